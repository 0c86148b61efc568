"""Pins of the oracle's FastSLS alternation (Sec. III-D, App. B)."""
import dataclasses

import numpy as np
import pytest

from oracle import fastsls, lq
from oracle import sls as osls
from paper_2604_07644_b300 import workloads as W


def test_tighten_moves_every_finite_bound_inwards():
    qp, sp = W.fastsls_problem(1)
    g = np.random.default_rng(0)
    h = g.uniform(0.0, 0.1, (qp.N, qp.nc))
    hf = g.uniform(0.0, 0.1, qp.nf)
    qt = fastsls.tighten(qp, h, hf)
    m = np.concatenate([h.ravel(), hf])
    fin_hi, fin_lo = np.isfinite(qp.hi), np.isfinite(qp.lo)
    assert np.allclose(qt.hi[fin_hi], qp.hi[fin_hi] - m[fin_hi], rtol=0, atol=0)
    assert np.allclose(qt.lo[fin_lo], qp.lo[fin_lo] + m[fin_lo], rtol=0, atol=0)
    assert np.all(np.isinf(qt.lo[~fin_lo])) and np.all(np.isinf(qt.hi[~fin_hi]))
    # stage k's block of rows uses h_k: row k*nc + c is moved by h[k, c]
    k, c = 5, 3
    assert qt.hi[k * qp.nc + c] == qp.hi[k * qp.nc + c] - h[k, c]


def test_first_step_uses_the_unweighted_controller():
    """With tau = None the controller update is eq. fastsls_qp with tau = 0:
    the Phi of the plain SLS solve."""
    qp, sp = W.fastsls_problem(2)
    s = fastsls.step(qp, sp, None)
    Px, Pu, h, hf, _ = osls.solve(dataclasses.replace(sp, tau=None))
    assert np.array_equal(s["Phix"], Px) and np.array_equal(s["h"], h)


def test_two_sided_row_equals_its_pair_of_one_sided_rows():
    """The |lambda| reading: a two-sided row lo <= g <= hi active at its
    lower bound (lambda < 0) is the one-sided row -g <= -lo with multiplier
    -lambda > 0 and the same row norm, so the SLS cost blocks of the pair
    (eq. sls_cost_matrices_tau) equal those of the two-sided row with
    tau = |lambda| / sqrt(beta + eps)."""
    qp, sp = W.fastsls_problem(1)
    Px, Pu, h, hf, _ = osls.solve(sp)
    g = np.random.default_rng(3)
    lam = g.standard_normal(qp.m)                  # both signs
    tau = fastsls.taus(sp, Px, Pu, lam)
    # the one-sided split: rows c and c' = -c, multipliers max(lam, 0) and max(-lam, 0)
    N, nc, nx = sp.N, sp.nc, sp.nx
    C2 = np.concatenate([sp.C, -sp.C], axis=1)
    D2 = np.concatenate([sp.D, -sp.D], axis=1)
    sp2 = dataclasses.replace(sp, C=C2, D=D2, CN=np.concatenate([sp.CN, -sp.CN]))
    lam_st = lam[:N * nc].reshape(N, nc)
    lam_tm = lam[N * nc:]
    lam2_st = np.concatenate([np.maximum(lam_st, 0), np.maximum(-lam_st, 0)], axis=1)
    lam2_tm = np.concatenate([np.maximum(lam_tm, 0), np.maximum(-lam_tm, 0)])
    tau2 = osls.beta_tau(sp2, Px, Pu, lam2_st, lam2_tm)
    for k, j in [(3, 1), (9, 4), (N - 1, 0)]:
        a = osls.cost_blocks(dataclasses.replace(sp, tau=tau), k, j)
        b = osls.cost_blocks(dataclasses.replace(sp2, tau=tau2), k, j)
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-12, atol=1e-12)
    a = osls.cost_blocks(dataclasses.replace(sp, tau=tau), N, 2)[0]
    b = osls.cost_blocks(dataclasses.replace(sp2, tau=tau2), N, 2)[0]
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def _disturbed_violation(qp, s, samples, seed=0, sign=1.0):
    """Largest violation of the ORIGINAL bounds by closed-loop trajectories
    x_k = x_k + sum_{j<k} Phi_x_{k,j} w_j, u_k = u_k + sum_{j<k} Phi_u_{k,j} w_j
    with |w_j|_2 <= 1 (the disturbance model of Sec. III-D), the nominal
    (x, u) of a step and its Phi."""
    g = np.random.default_rng(seed)
    N, nx, nu = qp.N, qp.nx, qp.nu
    worst = -np.inf
    for _ in range(samples):
        w = g.standard_normal((N, nx))
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        w *= g.uniform(0.5, 1.0, (N, 1))
        X = s["x"].copy()
        U = s["u"].copy()
        for k in range(1, N + 1):
            for j in range(k):
                X[k] += s["Phix"][(k - 1) * nx:k * nx, j * nx:(j + 1) * nx] @ w[j]
                if k < N:
                    U[k] += s["Phiu"][k * nu:(k + 1) * nu, j * nx:(j + 1) * nx] @ w[j]
        v = lq.G_apply(qp, X, U)
        worst = max(worst, float(np.max(np.maximum(v - qp.hi, qp.lo - v))))
    return worst


@pytest.mark.parametrize("seed", [1, 3])
def test_tightened_nominal_is_robustly_feasible(seed):
    """The point of the tightening: every disturbed closed-loop trajectory of
    a step stays inside the original bounds (Cauchy-Schwarz on each row), and
    some constraints are active, so the margins matter."""
    qp, sp = W.fastsls_problem(seed)
    hist = fastsls.alternation(qp, sp, 2)
    for s in hist:
        assert np.sum(np.abs(s["lam"]) > 1e-9) > 10
        assert _disturbed_violation(qp, s, 40) <= 1e-9


def test_planted_sign_error_in_the_tightening_is_caught():
    """Tightening outwards (lo - h, hi + h) instead of inwards lets disturbed
    trajectories leave the original bounds: the robust-feasibility pin fails."""
    qp, sp = W.fastsls_problem(1)
    orig = fastsls.tighten
    wrong = lambda q, h, hf: orig(q, -np.asarray(h), -np.asarray(hf))  # noqa: E731
    try:
        fastsls.tighten = wrong
        s = fastsls.step(qp, sp, None)
    finally:
        fastsls.tighten = orig
    assert _disturbed_violation(qp, s, 40) > 1e-3


def test_alternation_settles():
    """On a problem with active constraints the margins change less from
    step to step as the alternation proceeds."""
    qp, sp = W.fastsls_problem(1)
    hist = fastsls.alternation(qp, sp, 4)
    d = [np.max(np.abs(hist[i + 1]["h"] - hist[i]["h"])) for i in range(3)]
    assert d[2] < d[0]
    assert np.max(hist[-1]["tau"]) > 0
