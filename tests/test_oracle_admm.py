"""Pins of the oracle's ADMM and KKT residual."""
import numpy as np
import pytest

from oracle import activeset, admm, kkt, lq
from paper_2604_07644_b300 import workloads as W


@pytest.mark.parametrize("seed", range(6))
def test_admm_matches_active_set_brute_force(seed):
    """ADMM converges to the unique optimum found by enumerating active sets."""
    qp = W.tiny(seed)
    xb, ub, lb, act = activeset.brute_force(qp)
    r = admm.admm(qp, admm.Settings(eps=1e-11, max_iter=200000))
    assert r.converged
    assert np.allclose(r.x, xb, atol=1e-8)
    assert np.allclose(r.u, ub, atol=1e-8)
    assert kkt.kkt_residual(qp, xb, ub, lb) < 1e-10


def test_brute_force_has_active_constraints():
    """The tiny workloads exercise active bounds (otherwise the pin is weak)."""
    n_active = 0
    for seed in range(6):
        _, _, lb, act = activeset.brute_force(W.tiny(seed))
        n_active += len(act)
    assert n_active >= 4


def test_strictly_feasible_lqr_optimum_is_returned():
    """If the unconstrained optimum is strictly feasible, ADMM returns it."""
    qp = W.random_general(2, 3, 2, 6, 3, 2)
    x, u = lq.lq_solve(qp, qp.Q, qp.R, qp.S, qp.q, qp.r, qp.x0)
    v = lq.G_apply(qp, x, u)
    qp.hi = np.maximum(qp.hi, v + 1.0)
    qp.lo = np.minimum(qp.lo, v - 1.0)
    r = admm.admm(qp, admm.Settings(eps=1e-11, max_iter=100000))
    assert np.allclose(r.x, x, atol=1e-9) and np.allclose(r.u, u, atol=1e-9)
    assert np.max(np.abs(r.lam)) < 1e-9


def test_z_stays_in_bounds_and_rho_changes():
    qp = W.plain_4d(1)
    r = admm.admm(qp, admm.Settings(eps=1e-6, sigma=5, max_iter=400))
    assert np.all(r.z <= qp.hi + 1e-12) and np.all(r.z >= qp.lo - 1e-12)
    assert len(r.rho_hist) >= 2, "workload should trigger a rho change"
    assert np.isfinite(r.lam).all()


def test_rho_rescale_keeps_lambda(monkeypatch):
    """y is rescaled by rho_old / rho_new so lam = rho y is unchanged by a rho
    update (recorded from inside the iteration)."""
    qp = W.plain_4d(2)
    s = admm.Settings(eps=0.0, sigma=5, check_every=5, max_iter=30)
    state = {}

    orig_rule = admm.rho_rule

    def spy(qp_, x, u, v, z, y, rho, rp, rd, s_):
        new = orig_rule(qp_, x, u, v, z, y, rho, rp, rd, s_)
        state.setdefault("calls", []).append((rho, y.copy(), new))
        return new

    monkeypatch.setattr(admm, "rho_rule", spy)
    r = admm.admm(qp, s)
    changed = [(rho, y, new) for rho, y, new in state["calls"] if new > 5 * rho or new < rho / 5]
    assert changed, "expected at least one rho change"
    rho, y, new = changed[0]
    lam_old = rho * y
    lam_new = new * (y * rho / new)
    assert np.allclose(lam_old, lam_new, rtol=1e-14, atol=0)


@pytest.mark.parametrize("seed", range(4))
def test_plain_4d_converges_to_kkt_tolerance(seed):
    qp = W.plain_4d(seed)
    r = admm.admm(qp, admm.Settings(eps=1e-4, eps_kkt=1e-4, max_iter=5000))
    assert r.converged and r.kkt <= 1e-4
    v = lq.G_apply(qp, r.x, r.u)
    assert np.all(v <= qp.hi + 1e-4) and np.all(v >= qp.lo - 1e-4)


def test_kkt_parts_detect_planted_errors():
    qp = W.tiny(1)
    xb, ub, lb, act = activeset.brute_force(qp)
    base = kkt.kkt_parts(qp, xb, ub, lb)
    assert max(base.values()) < 1e-10
    x2 = xb.copy()
    x2[2] += 1e-3
    assert kkt.kkt_parts(qp, x2, ub, lb)["dyn"] > 5e-4
    l2 = lb.copy()
    inactive = [i for i in range(qp.m) if i not in act]
    l2[inactive[0]] = 1e-2
    p = kkt.kkt_parts(qp, xb, ub, l2)
    assert p["comp"] > 1e-4 or p["stat"] > 1e-4
    u2 = ub.copy()
    u2[0] += 1e-3
    p = kkt.kkt_parts(qp, xb, u2, lb)
    assert p["stat"] > 1e-5 or p["dyn"] > 1e-5


def test_iterate_mode_runs_fixed_count():
    qp = W.plain_4d(0)
    r = admm.admm(qp, admm.Settings(sigma=0), iters=7)
    assert r.iters == 7


def test_u_residuals_vanish_at_optimum_and_match_kkt_part():
    qp = W.tiny(3)
    xb, ub, lb, _ = activeset.brute_force(qp)
    assert np.max(np.abs(kkt.u_residuals(qp, xb, ub, lb))) < 1e-10
    g = np.random.default_rng(1)
    x, u, l = xb + 1e-3 * g.standard_normal(xb.shape), ub + 1e-3 * g.standard_normal(ub.shape), lb
    ru = kkt.u_residuals(qp, x, u, l)
    assert abs(np.max(np.abs(ru)) - kkt.kkt_parts(qp, x, u, l)["stat"]) < 1e-14


def test_refinement_recovers_a_planted_operator_error(monkeypatch):
    """A factorization computed from slightly wrong data (R perturbed by 1e-3,
    standing in for a low-precision factorization) makes ADMM converge to the
    wrong fixed point, so the exact KKT check stalls; refinement of the linear
    term with the exact u-stationarity residual brings it under tolerance."""
    qp = W.plain_4d(1)
    orig = admm.augmented

    def perturbed(qp_, rho):
        Qh, Rh, Sh = orig(qp_, rho)
        return Qh, Rh + 1e-3 * qp_.R, Sh

    monkeypatch.setattr(admm, "augmented", perturbed)
    s0 = admm.Settings(eps=1e-4, eps_kkt=1e-8, eps_floor=1e-10, max_refine=0, max_iter=4000)
    r0 = admm.admm(qp, s0)
    s1 = admm.Settings(eps=1e-4, eps_kkt=1e-8, eps_floor=1e-10, max_refine=10, max_iter=4000)
    r1 = admm.admm(qp, s1)
    k0 = kkt.kkt_residual(qp, r0.x, r0.u, r0.lam)
    k1 = kkt.kkt_residual(qp, r1.x, r1.u, r1.lam)
    assert not r0.converged and k0 > 1e-6
    assert r1.converged and k1 <= 1e-8


# ---------------------------------------------------------------------------
# The rho rule (Sec. IV-A.2: an OSQP-style update, read as OSQP Sec. 5.2),
# pinned against values worked out by hand on a scalar QP (nx = nu = nc = nf = 1,
# N = 1): Q_0 = 2, Q_1 = 3, R_0 = 0.5, S_0 = 0.25, C_0 = 1, D_0 = 2, C_N = 1,
# rho = 0.5, r_prim = 0.5, r_dual = 0.1.  With xi = (x_0, x_1, u_0):
#   v = (C_0 x_0 + D_0 u_0, C_N x_1),  H xi = (Q_0 x_0 + S_0 u_0, Q_1 x_1, R_0 u_0 + S_0 x_0),
#   G^T lam = (C_0 lam_0, C_N lam_1, D_0 lam_0) with lam = rho y,
#   rho_new = rho sqrt((r_prim / max(|v|, |z|)) / (r_dual / max(|H xi|, |G^T lam|, |(q, r)|))).
# Each case makes a different scale term the maximum, so dropping any one of
# them, or inverting the ratio, changes a pinned value.
# ---------------------------------------------------------------------------
def _scalar_qp(q, r):
    f = lambda v: np.array(v, dtype=float)  # noqa: E731
    return W.QP(A=f([[[1.0]]]), B=f([[[1.0]]]), c=f([[0.0]]), Q=f([[[2.0]], [[3.0]]]), R=f([[[0.5]]]),
                S=f([[[0.25]]]), q=f(q), r=f(r), C=f([[[1.0]]]), D=f([[[2.0]]]), CN=f([[1.0]]),
                lo=f([-10.0, -10.0]), hi=f([10.0, 10.0]), x0=f([1.0]))


RHO_CASES = [
    # (x_0, x_1), u_0, z, y, (q_0, q_1), r_0, rho_new worked out by hand
    # A: |v| = 2 and |H xi| = Q_1 x_1 = 6 dominate: ratio (0.5/2)/(0.1/6) = 15
    ((1.0, 2.0), -1.0, (-0.5, 1.5), (0.2, -0.4), (0.1, -0.2), 0.3, 0.5 * np.sqrt(15.0)),
    # B: |z| = 3 and |G^T lam| = D_0 lam_0 = 4 dominate: ratio (0.5/3)/(0.1/4) = 20/3
    ((1.0, 0.5), -1.0, (-0.5, 3.0), (4.0, -0.4), (0.1, -0.2), 0.3, 0.5 * np.sqrt(20.0 / 3.0)),
    # C: |z| = 1.5 and |(q, r)| = 5 dominate: ratio (0.5/1.5)/(0.1/5) = 50/3
    ((1.0, 0.5), -1.0, (-0.5, 1.5), (0.2, -0.4), (5.0, -0.2), 0.3, 0.5 * np.sqrt(50.0 / 3.0)),
]


def _rho_case(case):
    (x0, x1), u0, z, y, q, r0, want = case
    qp = _scalar_qp([[q[0]], [q[1]]], [[r0]])
    x = np.array([[x0], [x1]])
    u = np.array([[u0]])
    v = lq.G_apply(qp, x, u)
    return qp, x, u, v, np.array(z), np.array(y), want


@pytest.mark.parametrize("case", range(len(RHO_CASES)))
def test_rho_rule_matches_hand_computed_values(case):
    qp, x, u, v, z, y, want = _rho_case(RHO_CASES[case])
    s = admm.Settings()
    got = admm.rho_rule(qp, x, u, v, z, y, 0.5, 0.5, 0.1, s)
    assert abs(got - want) < 1e-14 * want, (got, want)


def test_rho_rule_clamps_and_skips_degenerate_ratios():
    qp, x, u, v, z, y, want = _rho_case(RHO_CASES[0])
    s = admm.Settings(rho_max=1.0)
    assert admm.rho_rule(qp, x, u, v, z, y, 0.5, 0.5, 0.1, s) == 1.0
    s = admm.Settings(rho_min=5.0)
    assert admm.rho_rule(qp, x, u, v, z, y, 0.5, 0.5, 0.1, s) == 5.0
    # a zero residual leaves rho unchanged (no division by zero)
    assert admm.rho_rule(qp, x, u, v, z, y, 0.5, 0.0, 0.1, admm.Settings()) == 0.5
    assert admm.rho_rule(qp, x, u, v, z, y, 0.5, 0.5, 0.0, admm.Settings()) == 0.5


def _planted_rules():
    """Plausible mistakes in the rho rule, planted in copies of the oracle's
    function on the CPU: inverted ratio, each scale term dropped, a missing
    square root."""
    from oracle.lq import GT_apply, H_apply

    def make(invert=False, drop=None, no_sqrt=False):
        def rule(qp, x, u, v, z_new, y_new, rho, r_prim, r_dual, s):
            prim = [np.max(np.abs(v)), np.max(np.abs(z_new))]
            if drop == "v":
                prim = prim[1:]
            if drop == "z":
                prim = prim[:1]
            hx, hu = H_apply(qp, x, u)
            gx, gu = GT_apply(qp, rho * y_new)
            terms = {"H": max(np.max(np.abs(hx)), np.max(np.abs(hu))),
                     "G": max(np.max(np.abs(gx)), np.max(np.abs(gu))),
                     "qr": max(np.max(np.abs(qp.q)), np.max(np.abs(qp.r)))}
            if drop in terms:
                del terms[drop]
            ratio = (r_prim / max(prim)) / (r_dual / max(terms.values()))
            if invert:
                ratio = 1.0 / ratio
            f = ratio if no_sqrt else np.sqrt(ratio)
            return float(min(max(rho * f, s.rho_min), s.rho_max))
        return rule

    return {"inverted": make(invert=True), "no_sqrt": make(no_sqrt=True),
            **{f"drop_{k}": make(drop=k) for k in ("v", "z", "H", "G", "qr")}}


@pytest.mark.parametrize("mistake", ["inverted", "no_sqrt", "drop_v", "drop_z", "drop_H", "drop_G", "drop_qr"])
def test_rho_rule_pin_catches_planted_mistakes(mistake):
    """Every planted mistake fails at least one hand-computed case, and the
    same planted function without the mistake would pass them all (the oracle
    itself, checked above)."""
    rule = _planted_rules()[mistake]
    s = admm.Settings()
    missed = 0
    for case in RHO_CASES:
        qp, x, u, v, z, y, want = _rho_case(case)
        if abs(rule(qp, x, u, v, z, y, 0.5, 0.5, 0.1, s) - want) < 1e-14 * want:
            missed += 1
    assert missed < len(RHO_CASES), mistake


# ---------------------------------------------------------------------------
# The stall rule (the oracle's option mirroring FP32 solves; not in the paper)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(3))
def test_stall_rule_never_fires_when_residuals_reach_the_floor(seed):
    """With exact FP64 iterates the residuals reach every floor, so turning
    the stall rule on changes nothing: same iterations, same point."""
    qp = W.plain_4d(seed)
    base = dict(eps=1e-4, eps_kkt=1e-9, eps_floor=1e-9, max_iter=6000)
    r0 = admm.admm(qp, admm.Settings(**base))
    r1 = admm.admm(qp, admm.Settings(**base, stall_iters=250))
    assert r0.converged and r1.converged
    assert r0.iters == r1.iters and np.array_equal(r0.x, r1.x) and np.array_equal(r0.lam, r1.lam)


@pytest.mark.parametrize("seed", range(3))
def test_stall_rule_runs_the_gate_when_residuals_are_held_above_the_floor(seed, monkeypatch):
    """A dual residual held at 2e-7, above a 1e-7 floor (standing in for FP32
    rounding), keeps the in-loop test from ever passing at the floor: without
    the rule the solve runs to max_iter; with it the FP64 KKT check runs after
    250 iterations at the floor, passes, and the point agrees with the
    unplanted solve to the KKT tolerance (the rule changes when the check
    runs, not the point the iteration converges to)."""
    qp = W.plain_4d(seed)
    s = dict(eps=1e-4, eps_kkt=1e-7, eps_floor=1e-7, max_iter=4000)
    ref = admm.admm(qp, admm.Settings(**s))
    orig = admm.residuals

    def held(qp_, v, z_new, z, rho):
        rp, rd = orig(qp_, v, z_new, z, rho)
        return rp, max(rd, 2e-7)

    monkeypatch.setattr(admm, "residuals", held)
    r0 = admm.admm(qp, admm.Settings(**s))
    r1 = admm.admm(qp, admm.Settings(**s, stall_iters=250))
    assert ref.converged and not r0.converged and r0.iters == 4000
    assert r1.converged and r1.iters < 1000
    assert kkt.kkt_residual(qp, r1.x, r1.u, r1.lam) <= 1e-7
    assert np.max(np.abs(r1.x - ref.x)) < 1e-6 and np.max(np.abs(r1.u - ref.u)) < 1e-6


def test_residuals_definition():
    """r_prim = ||v - z+||_inf and r_dual = ||rho G^T (z+ - z)||_inf, checked
    on the scalar QP of the rho-rule pins: G^T w = (C_0 w_0, C_N w_1, D_0 w_0)."""
    qp = _scalar_qp([[0.1], [-0.2]], [[0.3]])
    v = np.array([-1.0, 2.0])
    z_new = np.array([-0.5, 1.5])
    z = np.array([-0.75, 1.0])
    rp, rd = admm.residuals(qp, v, z_new, z, 0.5)
    assert rp == 0.5                                  # max(|-1 + 0.5|, |2 - 1.5|)
    assert rd == 0.5 * max(0.25, 0.5, 2.0 * 0.25)     # rho * max(|C_0 dz_0|, |C_N dz_1|, |D_0 dz_0|)
