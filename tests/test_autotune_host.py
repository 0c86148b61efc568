"""Host logic of the launch-shape autotuner (no GPU): buckets, keys,
candidate shapes, the solve-time model and the JSON cache."""
import copy

import pytest

from paper_2604_07644_b300 import autotune as AT
from paper_2604_07644_b300 import native


def test_buckets_are_smallest_covering_edge():
    assert AT.bucket(1, AT.NX_BUCKETS) == 16
    assert AT.bucket(16, AT.NX_BUCKETS) == 16
    assert AT.bucket(17, AT.NX_BUCKETS) == 32
    assert AT.bucket(61, AT.NX_BUCKETS) == 64
    assert AT.bucket(75, AT.NX_BUCKETS) == 80
    assert AT.bucket(5000, AT.B_BUCKETS) == 4096


def test_key_separates_precision_and_buckets():
    k = AT.key("B300", 1, 61, 100, 256)
    assert k == "B300|p1|nx64|N128|B256"
    assert AT.key("B300", 0, 61, 100, 256) != k
    assert AT.key("B300", 1, 61, 100, 255) == k          # same batch bucket


def test_candidates_respect_horizon():
    assert set(AT.candidates(3)) == {(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)}
    assert (8, 1) in AT.candidates(100)


def test_score_recovers_linear_model():
    # t(k) = 5 + 0.25 k: intercept 5, slope 0.25
    t = lambda k: 5.0 + 0.25 * k
    assert AT.score(t(10), t(40), 10, 40, 250) == pytest.approx(5.0 + 0.25 * 250)


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "tune.json")
    c = AT.Cache(p)
    assert c.get("x") is None
    c.put("x", AT.Choice(4, 1, 0.5))
    c2 = AT.Cache(p)
    assert c2.get("x") == AT.Choice(4, 1, 0.5)


def test_settings_copy_is_independent():
    s = native.default_settings()
    t = copy.copy(s)
    t.cluster = 3
    t.occupancy = 1
    assert s.cluster != 3 and s.occupancy == 0


def test_makespan_takes_the_slower_of_throughput_and_tail():
    # batch: 10 + 0.5 k for the whole batch; one QP: 2 + 0.2 k
    bt = (10 + 0.5 * 10, 10 + 0.5 * 40)
    ot = (2 + 0.2 * 10, 2 + 0.2 * 40)
    assert AT.makespan(bt, ot, 10, 40, 100, 200) == pytest.approx(10 + 50)        # throughput-bound
    assert AT.makespan(bt, ot, 10, 40, 100, 1000) == pytest.approx(2 + 200)       # tail-bound
