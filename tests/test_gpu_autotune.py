"""Autotuner on the GPU: it measures every launch shape that fits, caches the
winner, and the tuned settings solve to the same iterates as the defaults."""
import numpy as np
import pytest

from paper_2604_07644_b300 import autotune as AT
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W
from paper_2604_07644_b300.api import QPBatch

pytestmark = pytest.mark.gpu


def test_autotune_picks_cached_valid_shape(lib, tmp_path):
    qps = [W.quadrotor_12d(i, N=40) for i in range(8)]
    base = native.default_settings(precision=native.GPUSLS_FP32)
    cache = AT.Cache(str(tmp_path / "t.json"))
    ch = AT.tune(qps, base, expected_iters=100, k1=4, k2=12, cache=cache)
    assert (ch.cluster, ch.occupancy) in AT.candidates(40)
    assert ch.ms_per_qp > 0
    s, c2 = AT.choose(qps, base, cache=AT.Cache(str(tmp_path / "t.json")))   # served from the cache
    assert (c2.cluster, c2.occupancy) == (ch.cluster, ch.occupancy)
    assert s.cluster == ch.cluster and s.occupancy == ch.occupancy


@pytest.mark.parametrize("cluster,occ", [(1, 1), (4, 0), (8, 1)])
def test_launch_shapes_give_same_iterates(lib, cluster, occ):
    qps = [W.quadrotor_12d(3, N=40), W.random_general(2, 9, 3, 33, 6, 2)]
    ref = QPBatch(qps, native.default_settings(precision=native.GPUSLS_FP64, cluster=2, sigma=0, fixed_iters=15),
                  rho=0.3)
    r0 = ref.solve()
    s = native.default_settings(precision=native.GPUSLS_FP64, cluster=cluster, sigma=0, fixed_iters=15)
    s.occupancy = occ
    qb = QPBatch(qps, s, rho=0.3)
    r1 = qb.solve()
    for a, b in zip(r1.dx, r0.dx):
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.max(np.abs(b)))
    ref.close()
    qb.close()
