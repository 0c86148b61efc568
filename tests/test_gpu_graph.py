"""Serving graph (qp_graph_create / qp_graph_launch): one captured step of
reset, learned warm start and persistent solve gives, bit for bit, the results
of the same calls made one by one, and stays valid across replays and
problem updates."""
import os

import numpy as np
import pytest
import torch

from paper_2604_07644_b300 import learned, native
from paper_2604_07644_b300 import workloads as W
from paper_2604_07644_b300.api import QPBatch

pytestmark = pytest.mark.gpu

MODEL = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2604_07644_b300", "warmstart_quadruped61.npz")


def _snapshot(qb):
    return qb.out_x.clone(), qb.out_u.clone(), qb.out_l.clone()


def _eager(qb, mlp=None, feats=None):
    qb.reset()
    if mlp is not None:
        mlp.warm_start(qb, feats)
    r = qb.solve(fetch=True)
    return _snapshot(qb), r.info


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


def test_graph_cold_batch_matches_eager(lib):
    qps = [W.plain_4d(0), W.random_general(3, 7, 3, 23, 5, 2), W.quadrotor_12d(1, N=20)]
    st = native.default_settings(precision=native.GPUSLS_FP64, cluster=4)
    qb = QPBatch(qps, st)
    ref, info_e = _eager(qb)
    g = qb.graph()
    for _ in range(2):                       # replays are independent steps
        qb.out_x.zero_()
        g.launch()
        torch.cuda.synchronize()
        assert _same(_snapshot(qb), ref)
    info_g = g.info()
    for a, b in zip(info_g, info_e):
        assert a["iters"] == b["iters"] and a["status"] == b["status"] and a["kkt"] == b["kkt"]
    qb.close()


def test_graph_learned_warm_start_matches_eager(lib):
    fam = W.family(0)
    qps = [fam.instance(100000 + i) for i in range(6)]
    st = native.default_settings(precision=native.GPUSLS_FP32, cluster=8, max_refine=3, fallback_iters=2000,
                                 max_iter=6000, eps_floor=1e-5)
    qb = QPBatch(qps, st)
    mlp = learned.load(MODEL, max_batch=len(qps))
    feats = qb.features()            # the library's linearization features, given explicitly
    ref, info_e = _eager(qb, mlp, feats)
    g = qb.graph(mlp, feats)
    g.launch()
    torch.cuda.synchronize()
    assert _same(_snapshot(qb), ref)
    assert [i["iters"] for i in g.info()] == [i["iters"] for i in info_e]
    assert all(i["status"] == native.GPUSLS_OK for i in g.info())
    mlp.close()
    qb.close()


def test_graph_heads_match_eager_and_single_network(lib):
    """The per-family heads graph (features computed inside the graph) gives
    bit for bit the eager qp_warm_start_heads + solve, and the single-network
    path fed the same features."""
    fam = W.family(0)
    qps = [fam.instance(100010 + i) for i in range(6)]
    st = native.default_settings(precision=native.GPUSLS_FP32, cluster=8, max_refine=3, fallback_iters=2000,
                                 max_iter=6000, eps_floor=1e-5)
    qb = QPBatch(qps, st)
    mlp = learned.load(MODEL, max_batch=len(qps))
    heads = [(mlp, list(range(len(qps))), qps[0].N)]
    qb.reset()
    qb.warm_start_heads(heads)
    r = qb.solve(fetch=True)
    ref = _snapshot(qb)
    g = qb.graph(heads=heads)
    g.launch()
    torch.cuda.synchronize()
    assert _same(_snapshot(qb), ref)
    assert [i["iters"] for i in g.info()] == [i["iters"] for i in r.info]
    ref2, _ = _eager(qb, mlp, qb.features())
    assert _same(ref2, ref)
    mlp.close()
    qb.close()


def test_graph_sees_problem_updates_and_new_x0(lib):
    """Problem data changed by qp_update and x0 refilled in place between
    replays: the graph solves the new problem (equal to an eager solve)."""
    qps = [W.random_general(5, 6, 2, 17, 4, 2), W.random_general(6, 6, 2, 17, 4, 2)]
    st = native.default_settings(precision=native.GPUSLS_FP64, cluster=2)
    qb = QPBatch(qps, st)
    g = qb.graph()
    g.launch()
    torch.cuda.synchronize()
    gen = np.random.default_rng(7)
    new_q = [qp.q + 0.3 * gen.standard_normal(qp.q.shape) for qp in qps]
    new_x0 = [qp.x0 + 0.1 * gen.standard_normal(qp.x0.shape) for qp in qps]
    qb.update(q=new_q)
    qb.x0.copy_(torch.from_numpy(np.concatenate(new_x0)).to(qb.x0.device))
    g.launch()
    torch.cuda.synchronize()
    got = _snapshot(qb)
    # eager reference on a fresh handle with the updated problem
    for qp, q, x0 in zip(qps, new_q, new_x0):
        qp.q = q
        qp.x0 = x0
    qe = QPBatch(qps, st)
    ref, _ = _eager(qe)
    assert _same(got, ref)
    qe.close()
    qb.close()


def test_graph_rejects_null_arguments(lib):
    qb = QPBatch([W.tiny(0)])
    import ctypes as C
    g = C.c_void_p()
    st = lib.qp_graph_create(C.byref(g), qb.h, None, None, None, None, None, None, None, None, 1e-3, 1e3)
    assert st == native.GPUSLS_ERR_INVALID
    assert lib.qp_graph_launch(None, None) == native.GPUSLS_ERR_INVALID
    qb.close()


@pytest.mark.parametrize("graph", [False, True])
def test_longest_first_schedule_changes_only_the_order(lib, graph):
    """schedule = 1 launches the QPs longest-expected-first (from their own
    previous solve): every result, iteration count and status is the same as
    in index order, on every solve."""
    qps = [W.random_general(10 + i, 5 + i % 4, 2, 12 + 5 * i, 3, 1) for i in range(7)]
    s0 = native.default_settings(precision=native.GPUSLS_FP64, cluster=2)
    s1 = native.default_settings(precision=native.GPUSLS_FP64, cluster=2, schedule=1)
    q0, q1 = QPBatch(qps, s0), QPBatch(qps, s1)
    g1 = q1.graph() if graph else None
    for _ in range(3):
        ref, info0 = _eager(q0)
        if graph:
            g1.launch()
            torch.cuda.synchronize()
            got, info1 = _snapshot(q1), g1.info()
        else:
            got, info1 = _eager(q1)
        assert _same(got, ref)
        assert [i["iters"] for i in info1] == [i["iters"] for i in info0]
    q0.close()
    q1.close()


@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32])
def test_update_of_every_array_equals_a_fresh_handle(lib, prec):
    """qp_update of every problem array on a ragged batch (one device copy
    per array kind for the whole batch, pack jobs per QP): the next solve,
    its statuses, iteration counts and FP64 KKT residuals equal those of a
    handle set up from the new data."""
    keys = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi")
    old = [W.random_general(11, 6, 2, 17, 4, 2), W.random_general(12, 4, 3, 9, 0, 3),
           W.random_general(13, 7, 2, 23, 5, 0)]
    new = [W.random_general(21, 6, 2, 17, 4, 2), W.random_general(22, 4, 3, 9, 0, 3),
           W.random_general(23, 7, 2, 23, 5, 0)]
    for a, b in zip(old, new):
        b.x0 = a.x0.copy()   # x0 is not part of qp_update
    st = native.default_settings(precision=prec, cluster=2)
    qb = QPBatch(old, st)
    qb.solve()
    qb.update(**{k: [getattr(q, k) for q in new] for k in keys})
    qb.reset()
    r = qb.solve()
    got = _snapshot(qb)
    qb.close()
    qe = QPBatch(new, st)
    ref, info = _eager(qe)
    qe.close()
    assert _same(got, ref)
    assert [(i["status"], i["iters"], i["kkt"]) for i in r.info] == [(i["status"], i["iters"], i["kkt"]) for i in info]
