"""What the trained warm-start networks gain over the method without them,
on held-out instances (the networks were trained on instances 0..9999; these
are 100000+): the quadruped-shaped family of the headline and each shape
family of the serving mix (12D/4, 61D/12, 75D/21, ragged horizons), all from
the library's linearization features (qp_features) -- and that a warm start
that fails falls back to the cold method."""
import os

import numpy as np
import pytest
import torch

from oracle import kkt
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu

MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2604_07644_b300",
                     "warmstart_quadruped61.npz")


def test_learned_warm_start_gain(lib):
    from paper_2604_07644_b300 import learned
    from paper_2604_07644_b300.api import QPBatch
    fam = W.family(0)
    qps = [fam.instance(100000 + 500 + i) for i in range(64)]
    s = native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, max_refine=3, fallback_iters=1500)
    qb = QPBatch(qps, s)
    cold = qb.solve()
    mlp = learned.load(MODEL, max_batch=64)
    qb.reset()
    qb.warm_start_heads([(mlp, list(range(64)), qps[0].N)])
    warm = qb.solve()
    assert all(i["status"] == native.GPUSLS_OK for i in warm.info)
    ic = np.mean([i["iters"] for i in cold.info])
    iw = np.mean([i["iters"] for i in warm.info])
    rc = np.mean([i["refactors"] for i in cold.info])
    rw = np.mean([i["refactors"] for i in warm.info])
    print(f"held-out 64: iterations cold {ic:.1f} warm {iw:.1f}; refactors cold {rc:.2f} warm {rw:.2f}")
    assert iw < 0.95 * ic
    assert rw < 0.75 * rc
    for i in range(0, 64, 16):
        assert kkt.kkt_residual(qps[i], warm.dx[i], warm.du[i], warm.lam[i]) <= 1.0001e-4
    mlp.close()
    qb.close()


def test_bad_warm_start_falls_back_to_cold(lib):
    """A deliberately wrong warm start (huge multipliers, rho at its upper
    clamp) that has not converged by fallback_iters restarts cold and still
    returns the cold solution."""
    from paper_2604_07644_b300.api import QPBatch
    fam = W.family(0)
    qp = fam.instance(100777)
    s = native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, fallback_iters=50)
    qb = QPBatch([qp], s)
    cold = qb.solve()
    qb.reset()
    qb.set_warm_start([np.full(qp.m, 3.0)], [np.full(qp.m, 50.0)], 5e3)
    r = qb.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK
    assert np.max(np.abs(r.dx[0] - cold.dx[0])) < 1e-3
    qb.close()


def _rad_sign(salt, l, e):
    """The +-1 projection entries of qp_features, restated from their
    definition (a 32-bit mix of projection, row and input index)."""
    M = 0xFFFFFFFF
    h = ((salt * 0x9E3779B1) & M) ^ (((l + 0x7F4A7C15) * 0x85EBCA77) & M) ^ (((e + 0x165667B1) * 0xC2B2AE3D) & M)
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M
    h ^= h >> 16
    return 1.0 if h & 1 else -1.0


def _features_by_definition(qp, p=16):
    nx, nu, N, nc = qp.nx, qp.nu, qp.N, qp.nc
    mA = (qp.A.mean(axis=0) - np.eye(nx)).ravel()
    mB = qp.B.mean(axis=0).ravel()
    mq = qp.q.mean(axis=0)
    hs = qp.hi[:N * nc].reshape(N, nc)
    mh = np.where(np.isfinite(hs), np.clip(hs, -10, 10), 0.0).mean(axis=0) if nc else np.zeros(0)
    out = list(qp.x0)
    for salt, v in ((1, mA), (2, mB), (3, mq), (4, mh)):
        for l in range(p):
            s = sum(_rad_sign(salt, l, e) * v[e] for e in range(v.size))
            out.append(s / np.sqrt(v.size) if v.size else 0.0)
    # reorder: the kernel stores [x0, A (p), B (p), q (p), h (p), N / 128]
    return np.array(out + [N / 128.0])


def test_linearization_features_match_their_definition(lib):
    """qp_features on a ragged handle (12D, 61D, 75D QPs) equals the feature
    definition evaluated in numpy."""
    from paper_2604_07644_b300.api import QPBatch
    qps = [W.mix_family(0).instance(5, 40), W.family(0).instance(7), W.mix_family(2).instance(3, 25)]
    qb = QPBatch(qps, native.default_settings(precision=native.GPUSLS_FP32))
    F = qb.features().cpu().numpy()
    qb.close()
    for i, qp in enumerate(qps):
        want = _features_by_definition(qp)
        got = F[i, :want.size]
        assert np.max(np.abs(got - want)) <= 1e-4 * max(1.0, np.max(np.abs(want))), (i, np.max(np.abs(got - want)))
        assert np.all(F[i, want.size:] == 0.0)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_mix_family_head_gain(lib, kind):
    """Each shape family's head, on 64 held-out instances of ragged horizons
    (N ~ U{16..128}): fewer mean iterations than the cold start, every QP
    converged, sampled points pass the oracle's KKT check."""
    from paper_2604_07644_b300 import learned
    from paper_2604_07644_b300.api import QPBatch
    fam = W.mix_family(kind)
    Ns = [int(v) for v in W.rng(25, kind).integers(16, W.MIX_N_MAX + 1, 64)]
    qps = [fam.instance(100000 + i, N) for i, N in enumerate(Ns)]
    s = native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, max_refine=3, fallback_iters=1500,
                                max_iter=6000)
    qb = QPBatch(qps, s)
    cold = qb.solve()
    mlp = learned.load(os.path.join(os.path.dirname(MODEL), learned.MIX_MODELS[kind]), max_batch=64)
    qb.reset()
    qb.warm_start_heads([(mlp, list(range(64)), W.MIX_N_MAX)])
    warm = qb.solve()
    assert all(i["status"] == native.GPUSLS_OK for i in warm.info)
    ic = np.mean([i["iters"] for i in cold.info])
    iw = np.mean([i["iters"] for i in warm.info])
    print(f"family {kind}: iterations cold {ic:.1f} warm {iw:.1f}")
    assert iw < ic
    for i in range(0, 64, 16):
        assert kkt.kkt_residual(qps[i], warm.dx[i], warm.du[i], warm.lam[i]) <= 1.0001e-4
    mlp.close()
    qb.close()


def test_serving_mix_learned_graph(lib):
    """The 256-QP learned serving mix (three families, ragged nx and N) in one
    graph with a head per family: every QP converges and the mean iteration
    count is below the cold graph's on the same batch."""
    from paper_2604_07644_b300 import learned
    from paper_2604_07644_b300.api import QPBatch
    mix = W.serving_mix_learned(0, 256)
    qps = [q for q, _ in mix]
    s = native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, max_refine=3, fallback_iters=2000,
                                max_iter=6000, cluster=4)
    qb = QPBatch(qps, s)
    heads = learned.mix_heads(mix, os.path.dirname(MODEL))
    gw = qb.graph(heads=heads)
    gc = qb.graph()
    gc.launch()
    torch.cuda.synchronize()
    ic = np.mean([i["iters"] for i in gc.info()])
    gw.launch()
    torch.cuda.synchronize()
    info = gw.info()
    iw = np.mean([i["iters"] for i in info])
    print(f"serving mix: iterations cold {ic:.1f} learned {iw:.1f}")
    assert all(i["status"] == native.GPUSLS_OK for i in info)
    assert iw < ic
    for h in heads:
        h[0].close()
    qb.close()
