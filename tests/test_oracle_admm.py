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
