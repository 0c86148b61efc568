"""Pins of oracle.infeas (the primal infeasibility certificate) and of the
oracle ADMM's classification of solves that reach max_iter.

The recursion for the multipliers is checked against dense E and G built
here entry by entry from the QP's definition (eq. sqp_qp), so a sign or an
index error in it fails; the classification is checked on problems that are
infeasible by construction and on a feasible problem cut short."""
import numpy as np
import pytest

from oracle import admm, infeas
from paper_2604_07644_b300 import workloads as W


def dense_E_G(qp):
    """E, e of x_0 = x0 and x_{k+1} - A_k x_k - B_k u_k = c_k; G of the
    stage and terminal rows; xi = (x_0 .. x_N, u_0 .. u_{N-1})."""
    N, nx, nu, nc, nf = qp.N, qp.nx, qp.nu, qp.nc, qp.nf
    n = (N + 1) * nx + N * nu
    xi = lambda k: k * nx                      # noqa: E731
    ui = lambda k: (N + 1) * nx + k * nu       # noqa: E731
    E = np.zeros(((N + 1) * nx, n))
    e = np.zeros((N + 1) * nx)
    for a in range(nx):
        E[a, xi(0) + a] = 1.0
        e[a] = qp.x0[a]
    for k in range(N):
        for a in range(nx):
            row = (k + 1) * nx + a
            E[row, xi(k + 1) + a] = 1.0
            for b in range(nx):
                E[row, xi(k) + b] -= qp.A[k][a, b]
            for b in range(nu):
                E[row, ui(k) + b] -= qp.B[k][a, b]
            e[row] = qp.c[k][a]
    G = np.zeros((N * nc + nf, n))
    for k in range(N):
        for r in range(nc):
            for b in range(nx):
                G[k * nc + r, xi(k) + b] = qp.C[k][r, b]
            for b in range(nu):
                G[k * nc + r, ui(k) + b] = qp.D[k][r, b]
    for r in range(nf):
        for b in range(nx):
            G[N * nc + r, xi(N) + b] = qp.CN[r, b]
    return E, e, G


@pytest.mark.parametrize("make", [lambda: W.random_general(0, 3, 2, 5, 3, 2), lambda: W.random_general(1, 4, 3, 6, 2, 0),
                                  lambda: W.plain_4d(0, N=6)])
def test_multipliers_solve_the_x_components_of_the_dense_system(make):
    qp = make()
    rng = np.random.default_rng(7)
    w = rng.standard_normal(qp.m)
    nu_, mu0, r = infeas.multipliers(qp, w)
    E, e, G = dense_E_G(qp)
    mu = np.concatenate([mu0, nu_.reshape(-1)])
    g = E.T @ mu + G.T @ w
    nxs = (qp.N + 1) * qp.nx
    assert np.max(np.abs(g[:nxs])) < 1e-12 * max(1.0, np.max(np.abs(w)))
    assert np.allclose(g[nxs:], r.reshape(-1), atol=1e-12)
    # the certificate's value is sigma(w) + e^T mu, summed densely
    sig = sum((h * wi if wi > 0 else lo * wi) for wi, lo, h in zip(w, qp.lo, qp.hi)
              if (wi > 0 and np.isfinite(h)) or (wi < 0 and np.isfinite(lo)))
    c = infeas.certificate(qp, w, 1e-4)
    assert abs(c["value"] - (sig + e @ mu)) < 1e-10 * max(1.0, abs(c["value"]))


@pytest.mark.parametrize("make", [W.infeasible_x0, W.infeasible_terminal])
def test_infeasible_problems_are_certified_at_max_iter(make):
    qp = make()
    r = admm.admm(qp, admm.Settings(max_iter=600))
    assert not r.converged and r.infeasible
    # and the direction is a certificate in the exact sense: the value is
    # negative by more than the residual can explain
    w_dir = r.lam / max(1.0, np.max(np.abs(r.lam)))
    c = infeas.certificate(qp, w_dir, 1e-3)
    assert c["value"] < 0.0


def test_feasible_problem_cut_short_is_not_certified():
    qp = W.plain_4d(0)
    r = admm.admm(qp, admm.Settings(max_iter=20))
    assert not r.converged and not r.infeasible


def test_planted_sign_error_in_the_recursion_is_caught():
    """A flipped C^T w term in the recursion no longer solves the dense
    x-components (the pin above would fail)."""
    qp = W.random_general(0, 3, 2, 5, 3, 2)
    w = np.random.default_rng(3).standard_normal(qp.m)
    nu_, mu0, r = infeas.multipliers(qp, w)
    bad = nu_.copy()
    wk = w[:qp.N * qp.nc].reshape(qp.N, qp.nc)
    for k in range(qp.N - 1, 0, -1):
        bad[k - 1] = qp.A[k].T @ bad[k] + qp.C[k].T @ wk[k]
    E, e, G = dense_E_G(qp)
    g = E.T @ np.concatenate([mu0, bad.reshape(-1)]) + G.T @ w
    assert np.max(np.abs(g[:(qp.N + 1) * qp.nx])) > 1e-6
