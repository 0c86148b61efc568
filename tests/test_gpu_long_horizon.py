"""Long horizons (Sec. V-A's horizon study, N up to 3000): the torque-limited
pendulum-shaped workload (nx=30, nu=15, N=3000, 1.35e5 decision variables),
whose per-chunk vectors no longer fit a CTA's shared memory and live in a
per-CTA global region (at 8 CTAs per QP, and at 16, a non-portable cluster
size that halves the chunks), against the FP64 oracle: the factorization against
the sequential Riccati recursion, iterates against the step-by-step ADMM,
and an adaptive FP32 solve against the oracle's KKT measure.  The global-
region path is also compared with the shared-memory path on a horizon both
can run."""
import numpy as np
import pytest

from oracle import admm, kkt, lq
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def batch(qps, **kw):
    from paper_2604_07644_b300.api import QPBatch
    rho = kw.pop("rho", None)
    return QPBatch(qps, native.default_settings(**kw), rho=rho)


@pytest.fixture(scope="module")
def pend():
    return W.long_horizon(0)


@pytest.mark.parametrize("cluster", [8, 16])
@pytest.mark.parametrize("prec,tol", [(native.GPUSLS_FP64, 1e-8), (native.GPUSLS_FP32, 1e-4)])
def test_riccati_matches_sequential_recursion_N3000(lib, pend, prec, tol, cluster):
    qp = pend
    rho = 0.5
    b = batch([qp], precision=prec, cluster=cluster, rho=rho)
    Ps, Ks = b.riccati()
    b.close()
    Qh, Rh, Sh = lq.augmented(qp, rho)
    P, p, K, kff, G = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, np.zeros_like(qp.q), np.zeros_like(qp.r))
    assert rel(Ps[0], P) < tol, rel(Ps[0], P)
    assert rel(Ks[0], K) < tol, rel(Ks[0], K)


@pytest.mark.parametrize("cluster", [8, 16])
def test_fixed_iterations_match_oracle_N3000(lib, pend, cluster):
    qp = pend
    b = batch([qp], precision=native.GPUSLS_FP64, cluster=cluster, sigma=0, fixed_iters=5, rho=0.1)
    r = b.solve()
    b.close()
    o = admm.admm(qp, admm.Settings(rho0=0.1, sigma=0), iters=5)
    assert rel(r.dx[0], o.x) < 1e-9 and rel(r.du[0], o.u) < 1e-9 and rel(r.lam[0], o.lam) < 1e-9


@pytest.mark.parametrize("cluster", [8, 16])
def test_adaptive_fp32_solve_N3000(lib, pend, cluster):
    """The solve to the 1e-4 KKT tolerance: the returned point passes the
    oracle's KKT check and meets every torque limit."""
    qp = pend
    b = batch([qp], precision=native.GPUSLS_FP32, cluster=cluster, eps_floor=1e-5, max_iter=20000)
    r = b.solve()
    b.close()
    assert r.info[0]["status"] == native.GPUSLS_OK, r.info[0]
    assert kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0]) <= 1.0001e-4
    v = lq.G_apply(qp, r.dx[0], r.du[0])
    assert np.all(v <= qp.hi + 1e-4) and np.all(v >= qp.lo - 1e-4)
    assert np.max(np.abs(r.lam[0])) > 0.0          # torque limits active


@pytest.mark.parametrize("prec,tol", [(native.GPUSLS_FP64, 1e-9), (native.GPUSLS_FP32, 1e-4)])
def test_global_vectors_match_shared_vectors(lib, prec, tol):
    """A 6-link pendulum-shaped QP at N = 1024 (nx=12, nu=6): at cluster 1
    its per-chunk vectors (1024 stages, ~0.75 MB in FP64) go to the global
    region; at cluster 8 (128 stages per chunk) they stay in shared memory.
    Both match the oracle's iterates and each other.  (A quadrotor-shaped
    QP at this horizon is no test of the kernel: its closed loop is not
    contractive and the oracle's own FP64 Riccati recursion drifts 5e-7 from
    an extended-precision one there.)"""
    qp = W.long_horizon(1, links=6, N=1024)
    o = admm.admm(qp, admm.Settings(rho0=0.2, sigma=0), iters=7)
    out = {}
    for cs in (1, 8):
        b = batch([qp], precision=prec, cluster=cs, sigma=0, fixed_iters=7, rho=0.2)
        r = b.solve()
        b.close()
        assert rel(r.dx[0], o.x) < tol and rel(r.lam[0], o.lam) < tol, (cs, rel(r.dx[0], o.x))
        out[cs] = r.dx[0]
    assert rel(out[1], out[8]) < (1e-12 if prec == native.GPUSLS_FP64 else 1e-5)


def test_automatic_launch_shape_takes_16_cta_clusters_N3000(lib, pend):
    """With cluster = 0 a horizon whose 8-CTA chunks would need the global
    vector region runs in clusters of 16 CTAs (non-portable): its iterates
    are bit-identical to an explicit cluster-16 solve and differ, by
    rounding only, from the 8-CTA chunking."""
    out = {}
    for cs in (0, 16, 8):
        b = batch([pend], precision=native.GPUSLS_FP32, cluster=cs, sigma=0, fixed_iters=20, rho=0.1)
        out[cs] = b.solve().dx[0].copy()
        b.close()
    assert np.array_equal(out[0], out[16])
    assert not np.array_equal(out[0], out[8])
    assert rel(out[0], out[8]) < 1e-4
