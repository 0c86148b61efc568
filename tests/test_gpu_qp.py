"""GPU parity of the ADMM QP path against the FP64 oracle (calls through the
C ABI).  Tolerances: 1e-6 relative in FP64, 1e-4 relative in FP32 (relative
to max(1, max |reference|))."""
import numpy as np
import pytest

from oracle import activeset, admm, kkt, lq
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {native.GPUSLS_FP64: 1e-6, native.GPUSLS_FP32: 1e-4, native.GPUSLS_MIXED: 1e-4}


def rel(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b))))) if b.size else 0.0


def batch(qps, **kw):
    from paper_2604_07644_b300.api import QPBatch
    rho = kw.pop("rho", None)
    return QPBatch(qps, native.default_settings(**kw), rho=rho)


CASES = [
    ("tiny", lambda: W.tiny(0)),
    ("general-3-2-5", lambda: W.random_general(0, 3, 2, 5, 3, 2)),
    ("general-7-3-23", lambda: W.random_general(1, 7, 3, 23, 5, 0)),
    ("general-12-4-37-nc0", lambda: W.random_general(2, 12, 4, 37, 0, 3)),
    ("plain4d", lambda: W.plain_4d(0)),
    ("quad12d-N64", lambda: W.quadrotor_12d(0)),
]


@pytest.mark.parametrize("fact", [0, 1])
@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32, native.GPUSLS_MIXED])
@pytest.mark.parametrize("cluster", [1, 3, 8, 16])
@pytest.mark.parametrize("name,make", CASES)
def test_riccati_matches_oracle(lib, name, make, cluster, prec, fact):
    """The refactor (eq. assoc_init, eq. combination_rules, eq.
    controller_cache) gives the sequential Riccati P_i and K_i, with the
    blocked schedule (fact 0: leaf-structured combines, chunk elements
    combined across the cluster) and with the tree (fact 1)."""
    qp = make()
    rho = 0.7
    b = batch([qp], precision=prec, cluster=cluster, rho=rho, factorization=fact)
    Ps, Ks = b.riccati()
    Qh, Rh, Sh = lq.augmented(qp, rho)
    P, p, K, kff, G = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, np.zeros_like(qp.q), np.zeros_like(qp.r))
    tol = TOL[prec] * (1e-2 if prec == native.GPUSLS_FP64 else 10)
    assert rel(Ps[0], P) < tol, rel(Ps[0], P)
    assert rel(Ks[0], K) < tol, rel(Ks[0], K)
    b.close()


@pytest.mark.parametrize("cluster", [1, 2, 5, 8, 16])
@pytest.mark.parametrize("name,make", CASES)
def test_fixed_iterations_match_oracle_fp64(lib, name, make, cluster):
    """Iterate parity: 9 ADMM iterations at fixed rho from a cold start."""
    qp = make()
    b = batch([qp], precision=native.GPUSLS_FP64, cluster=cluster, sigma=0, fixed_iters=9, rho=0.3)
    r = b.solve()
    o = admm.admm(qp, admm.Settings(rho0=0.3, sigma=0), iters=9)
    assert rel(r.dx[0], o.x) < 1e-9
    assert rel(r.du[0], o.u) < 1e-9
    assert rel(r.lam[0], o.lam) < 1e-9
    assert r.info[0]["iters"] == 9
    b.close()


@pytest.mark.parametrize("prec", [native.GPUSLS_FP32, native.GPUSLS_MIXED])
@pytest.mark.parametrize("name,make", CASES)
def test_fixed_iterations_match_oracle_fp32(lib, name, make, prec):
    qp = make()
    b = batch([qp], precision=prec, sigma=0, fixed_iters=9, rho=0.3)
    r = b.solve()
    o = admm.admm(qp, admm.Settings(rho0=0.3, sigma=0), iters=9)
    assert rel(r.dx[0], o.x) < 1e-4
    assert rel(r.du[0], o.u) < 1e-4
    assert rel(r.lam[0], o.lam) < 1e-4
    b.close()


@pytest.mark.parametrize("seed", range(4))
def test_solution_matches_brute_force_tiny(lib, seed):
    """Converged solution equals the active-set brute-force optimum."""
    qp = W.tiny(seed)
    xb, ub, lb, _ = activeset.brute_force(qp)
    b = batch([qp], precision=native.GPUSLS_FP64, eps=1e-10, eps_kkt=1e-9, max_iter=100000)
    r = b.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK
    assert rel(r.dx[0], xb) < 1e-6 and rel(r.du[0], ub) < 1e-6
    b.close()


@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32])
@pytest.mark.parametrize("seed", range(3))
def test_adaptive_solve_plain4d(lib, seed, prec):
    """Adaptive-rho solve to the 1e-4 KKT tolerance: the returned point passes
    the oracle's own KKT check, satisfies every bound, and matches the exact
    optimum."""
    qp = W.plain_4d(seed)
    b = batch([qp], precision=prec)
    r = b.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK
    k_or = kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0])
    assert k_or <= 1.0001e-4
    v = lq.G_apply(qp, r.dx[0], r.du[0])
    assert np.all(v <= qp.hi + 1e-4) and np.all(v >= qp.lo - 1e-4)
    assert abs(r.info[0]["kkt"] - k_or) <= 1e-12 + 1e-9 * k_or
    o = admm.admm(qp, admm.Settings(eps=1e-4, eps_kkt=1e-4))
    if prec == native.GPUSLS_FP64:
        assert r.info[0]["iters"] == o.iters
        assert rel(r.dx[0], o.x) < 1e-6
    b.close()


def test_kkt_entry_point_matches_oracle(lib):
    qp = W.tiny(2)
    xb, ub, lb, _ = activeset.brute_force(qp)
    g = np.random.default_rng(0)
    b = batch([qp])
    for pert in [0.0, 1e-3]:
        x = xb + pert * g.standard_normal(xb.shape)
        u = ub + pert * g.standard_normal(ub.shape)
        l = lb + pert * g.standard_normal(lb.shape)
        got = b.kkt([x], [u], [l])[0]
        assert abs(got - kkt.kkt_residual(qp, x, u, l)) < 1e-12 + 1e-9 * abs(got)
    b.close()


def test_batch_equals_single(lib):
    """A ragged batch gives, QP by QP, the single-instance results."""
    qps = [W.random_general(5, 3, 2, 11, 2, 1), W.plain_4d(1), W.random_general(6, 9, 4, 30, 6, 2),
           W.quadrotor_12d(1, N=20)]
    bb = batch(qps, precision=native.GPUSLS_FP64, sigma=0, fixed_iters=12, rho=0.5, cluster=4)
    rb = bb.solve()
    for i, qp in enumerate(qps):
        bs = batch([qp], precision=native.GPUSLS_FP64, sigma=0, fixed_iters=12, rho=0.5, cluster=4)
        rs = bs.solve()
        assert rel(rb.dx[i], rs.dx[0]) < 1e-12
        assert rel(rb.lam[i], rs.lam[0]) < 1e-12
        bs.close()
    bb.close()


def test_warm_start_state_roundtrip_and_resume(lib):
    """qp_get_state / qp_set_warm_start: resuming from a saved state equals
    running the iterations in one go (checkpoint / resume of the ADMM state)."""
    qp = W.plain_4d(2)
    b1 = batch([qp], sigma=0, fixed_iters=10, rho=0.4)
    r1 = b1.solve()
    z, y, rho = b1.get_state()
    r1b = b1.solve()                     # 10 more
    b2 = batch([qp], sigma=0, fixed_iters=10, rho=0.4)
    b2.set_warm_start(z, y, rho)
    r2 = b2.solve()
    assert rel(r2.dx[0], r1b.dx[0]) < 1e-12 and rel(r2.lam[0], r1b.lam[0]) < 1e-12
    o = admm.admm(qp, admm.Settings(rho0=0.4, sigma=0), iters=20)
    assert rel(r2.dx[0], o.x) < 1e-9
    b1.close()
    b2.close()


def test_unconstrained_rows_give_lqr(lib):
    """Loose bounds: the solution is the LQR optimum and lambda = 0."""
    qp = W.random_general(3, 5, 2, 17, 4, 2)
    x, u = lq.lq_solve(qp, qp.Q, qp.R, qp.S, qp.q, qp.r, qp.x0)
    v = lq.G_apply(qp, x, u)
    qp.hi = np.maximum(qp.hi, v + 1.0)
    qp.lo = np.minimum(qp.lo, v - 1.0)
    b = batch([qp], eps=1e-10, eps_kkt=1e-9)
    r = b.solve()
    assert rel(r.dx[0], x) < 1e-7 and rel(r.du[0], u) < 1e-7
    assert np.max(np.abs(r.lam[0])) < 1e-7
    b.close()


def test_quadruped_61d_full_size(lib):
    """Full-size 61D / N=100 QP: iterate parity for 6 fixed iterations in FP64,
    and the adaptive FP32 solve reaches the 1e-4 KKT tolerance by the oracle's
    own KKT measure with every constraint satisfied."""
    qp = W.quadruped_61d(0)
    b = batch([qp], precision=native.GPUSLS_FP64, sigma=0, fixed_iters=6, rho=0.1)
    r = b.solve()
    o = admm.admm(qp, admm.Settings(rho0=0.1, sigma=0), iters=6)
    assert rel(r.dx[0], o.x) < 1e-6 and rel(r.lam[0], o.lam) < 1e-6
    b.close()
    b = batch([qp], precision=native.GPUSLS_FP32)
    r = b.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK
    assert kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0]) <= 1.0001e-4
    v = lq.G_apply(qp, r.dx[0], r.du[0])
    assert np.all(v <= qp.hi + 1e-4) and np.all(v >= qp.lo - 1e-4)
    b.close()


@pytest.mark.parametrize("cluster", [6, 8])
def test_fp64_adaptive_solve_full_size(lib, cluster):
    """Full-size 61D / N=100 adaptive FP64 solve (rho updates every sigma
    iterations, checks, the KKT gate): the whole-region copies of the
    chunk-boundary corrections, of Sig_i and Q_i (rho rule) and of the [C D]
    blocks (dual residual) take several rounds per run in FP64.  The solution
    meets the 1e-4 tolerance by the oracle's own KKT measure with every
    constraint satisfied."""
    qp = W.quadruped_61d(1)
    b = batch([qp], precision=native.GPUSLS_FP64, cluster=cluster)
    r = b.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK
    assert r.info[0]["iters"] > 25   # at least one rho evaluation ran
    assert kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0]) <= 1.0001e-4
    v = lq.G_apply(qp, r.dx[0], r.du[0])
    assert np.all(v <= qp.hi + 1e-4) and np.all(v >= qp.lo - 1e-4)
    b.close()


@pytest.mark.parametrize("cluster", [6, 8])
def test_riccati_schedules_agree_full_size(lib, cluster):
    """Full-size 61D / N=100 factorization at the tuned launch shapes: the
    blocked schedule (leaf-structured combines) and the tree give the same
    P_i and K_i in FP64, and the FP32 blocked terms match the FP64 oracle's
    sequential Riccati recursion."""
    qp = W.quadruped_61d(0)
    rho = 0.3
    out = {}
    for fact in (0, 1):
        b = batch([qp], precision=native.GPUSLS_FP64, cluster=cluster, rho=rho, factorization=fact)
        out[fact] = b.riccati()
        b.close()
    assert rel(out[0][0][0], out[1][0][0]) < 1e-12
    assert rel(out[0][1][0], out[1][1][0]) < 1e-12
    Qh, Rh, Sh = lq.augmented(qp, rho)
    P, p, K, kff, G = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, np.zeros_like(qp.q), np.zeros_like(qp.r))
    assert rel(out[0][0][0], P) < 1e-8 and rel(out[0][1][0], K) < 1e-8
    b = batch([qp], precision=native.GPUSLS_FP32, cluster=cluster, rho=rho)
    Ps, Ks = b.riccati()
    b.close()
    assert rel(Ps[0], P) < 1e-4 and rel(Ks[0], K) < 1e-4


def test_fp32_stall_rule_converges(lib):
    """A 75D QP of the serving mix whose FP32 dual residual stays just above
    the 1e-5 eps floor: the stall rule runs the FP64 KKT gate (and refines)
    instead of iterating to max_iter."""
    qp = W.serving_mix(0, 256)[11]
    b = batch([qp], precision=native.GPUSLS_FP32, cluster=8, max_refine=3, max_iter=6000)
    r = b.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK, r.info[0]
    assert r.info[0]["iters"] < 6000 and r.info[0]["kkt"] <= 1e-4
    assert kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0]) <= 1.0001e-4
    b.close()


def test_cluster_sizes_give_the_same_fp64_iterates(lib):
    """The cluster sizes the autotuner can pick at this size run the same
    ADMM: 6 fixed FP64 iterations on the 61D problem agree to 1e-9."""
    qp = W.quadruped_61d(0)
    ref = None
    for cs in (4, 5, 6, 7, 8):   # shared memory per CTA limits FP64 at N = 100 to the larger clusters
        b = batch([qp], precision=native.GPUSLS_FP64, cluster=cs, sigma=0, fixed_iters=6, rho=0.1)
        r = b.solve()
        if ref is None:
            ref = r.dx[0].copy()
        assert rel(r.dx[0], ref) < 1e-9, cs
        b.close()


def test_invalid_dims_rejected(lib):
    qp = W.random_general(0, 3, 2, 5, 2, 1)
    qp.A = np.zeros((5, 81, 81))
    with pytest.raises(RuntimeError):
        batch([qp])


def test_fp32_refinement_reaches_kkt_on_stalling_instance(lib):
    """A held-out family instance whose FP32 fixed point stalls at a KKT of
    ~1e-4 (u-stationarity) converges once the iterative refinement of the
    linear term is allowed; the returned point passes the oracle's KKT check."""
    fam = W.family(0)
    qp = fam.instance(100094)
    b = batch([qp], precision=native.GPUSLS_FP32, eps_floor=1e-5, max_refine=3)
    r = b.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK, r.info
    assert kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0]) <= 1.0001e-4
    b.close()
    b = batch([qp], precision=native.GPUSLS_FP32, eps_floor=1e-5, max_refine=3)
    b.reset()
    r2 = b.solve()
    assert r2.info[0]["iters"] == r.info[0]["iters"]   # reset undoes the corrections
    b.close()


@pytest.mark.parametrize("name,make", [("plain4d", lambda: W.plain_4d(1)), ("quad12d", lambda: W.quadrotor_12d(2)),
                                       ("quadruped61", lambda: W.quadruped_61d(0))])
def test_tf32_products_accuracy_level(lib, name, make):
    """GPUSLS_TF32 (factorization block products in TF32 on the tensor cores,
    one pass): the Riccati terms carry the TF32 product error (a few 1e-3,
    checked against the oracle), and the FP64 KKT gate certifies what that
    operator allows: a 3e-3 KKT tolerance is reached with every bound
    satisfied to it.  (1e-4 is not reachable in this mode: the refinement of
    the linear term cannot undo a 1e-3 operator error.)"""
    qp = make()
    b = batch([qp], precision=native.GPUSLS_TF32, rho=0.5)
    Ps, Ks = b.riccati()
    Qh, Rh, Sh = lq.augmented(qp, 0.5)
    P, p, K, kff, G = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, np.zeros_like(qp.q), np.zeros_like(qp.r))
    assert 1e-5 < rel(Ps[0], P) < 1e-2          # TF32-sized error, not FP32-sized
    assert rel(Ks[0], K) < 1e-2
    b.close()
    b = batch([qp], precision=native.GPUSLS_TF32, max_refine=8, max_iter=8000)
    r = b.solve(tol=3e-3)
    assert r.info[0]["status"] == native.GPUSLS_OK, r.info
    assert kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0]) <= 3.0001e-3
    v = lq.G_apply(qp, r.dx[0], r.du[0])
    assert np.all(v <= qp.hi + 3e-3) and np.all(v >= qp.lo - 3e-3)
    b.close()


@pytest.mark.parametrize("cluster", [6, 8])
def test_mixed_precision_full_size(lib, cluster):
    """GPUSLS_MIXED at 61D / N=100 (block products in three TF32 passes on the
    tensor cores, per-stage solves to FP64 accuracy): the Riccati terms carry FP32-sized
    errors against the FP64 sequential recursion (1e-4 relative, like FP32,
    where one TF32 pass leaves 2e-3 to 5e-3), and the adaptive solve meets the
    1e-4 KKT tolerance by the oracle's own measure with every bound met."""
    qp = W.quadruped_61d(0)
    rho = 0.3
    b = batch([qp], precision=native.GPUSLS_MIXED, cluster=cluster, rho=rho)
    Ps, Ks = b.riccati()
    b.close()
    Qh, Rh, Sh = lq.augmented(qp, rho)
    P, p, K, kff, G = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, np.zeros_like(qp.q), np.zeros_like(qp.r))
    assert rel(Ps[0], P) < 1e-4 and rel(Ks[0], K) < 1e-4, (rel(Ps[0], P), rel(Ks[0], K))
    b = batch([qp], precision=native.GPUSLS_MIXED, cluster=cluster)
    r = b.solve()
    b.close()
    assert r.info[0]["status"] == native.GPUSLS_OK
    assert kkt.kkt_residual(qp, r.dx[0], r.du[0], r.lam[0]) <= 1.0001e-4
    v = lq.G_apply(qp, r.dx[0], r.du[0])
    assert np.all(v <= qp.hi + 1e-4) and np.all(v >= qp.lo - 1e-4)


def ill_conditioned_nodes(seed=0, nx=6, nu=4, N=12, small=1e-4):
    """A QP whose node blocks Gamma_i = R^_i + B_i^T P_{i+1} B_i have condition
    numbers 3e4..1e5: R_i has the eigenvalue `small` along a rotated input
    direction v, B_i and D_i nearly miss v, and S_i = 0 keeps each stage cost
    convex."""
    import dataclasses
    qp = W.random_general(seed, nx, nu, N, 3, 2)
    rng = np.random.default_rng(100 + seed)
    V, _ = np.linalg.qr(rng.standard_normal((nu, nu)))
    v = V[:, 0]
    R = V @ np.diag([small] + [1.0] * (nu - 1)) @ V.T
    Pv = np.eye(nu) - np.outer(v, v)
    return dataclasses.replace(qp, R=np.repeat(R[None], N, 0), S=np.zeros_like(qp.S),
                               B=qp.B @ Pv + 1e-3 * (qp.B @ np.outer(v, v)), D=qp.D @ Pv)


@pytest.mark.parametrize("cluster", [1, 3])
def test_mixed_node_solve_ill_conditioned(lib, cluster):
    """Node blocks of condition 3e4..1e5: the FP32 inverse's residual
    ||I - Gamma X0||_inf exceeds the refined node solve's 1e-4 threshold
    (numpy's pivoted FP32 inverse of these blocks leaves 2.5e-4..1.8e-3), so
    GPUSLS_MIXED takes its FP64 elimination for them.  P_i and K_i match the
    FP64 sequential recursion at least as well as the FP32 path does."""
    qp = ill_conditioned_nodes()
    rho = 0.7
    Qh, Rh, Sh = lq.augmented(qp, rho)
    P, p, K, kff, G = lq.riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, np.zeros_like(qp.q), np.zeros_like(qp.r))
    assert min(np.linalg.cond(np.linalg.inv(g)) for g in G) > 1e4
    err = {}
    for prec in (native.GPUSLS_FP32, native.GPUSLS_MIXED):
        b = batch([qp], precision=prec, cluster=cluster, rho=rho)
        Ps, Ks = b.riccati()
        b.close()
        assert np.all(np.isfinite(Ps[0])) and np.all(np.isfinite(Ks[0]))
        err[prec] = (rel(Ps[0], P), rel(Ks[0], K))
    eP, eK = err[native.GPUSLS_MIXED]
    fP, fK = err[native.GPUSLS_FP32]
    assert eP < 1e-3 and eK < 1e-2, err
    assert eK <= 2.0 * fK + 1e-5 and eP <= 2.0 * fP + 1e-5, err
