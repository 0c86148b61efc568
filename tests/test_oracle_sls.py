"""Pins of the oracle's SLS solve and margins (Sec. III-D, IV-B)."""
import numpy as np
import pytest

from oracle import lq, scan, sls
from paper_2604_07644_b300 import workloads as W


def _column_problem(sp, j, col):
    """The j-th controller problem restricted to column col: an LQR from the
    state E_j e_col at time j+1 over stages j+1..N-1 with costs Q_{k,j}."""
    N = sp.N
    ks = list(range(j + 1, N))
    n = len(ks)
    A = np.stack([sp.A[k] for k in ks]) if n else np.zeros((0, sp.nx, sp.nx))
    B = np.stack([sp.B[k] for k in ks]) if n else np.zeros((0, sp.nx, sp.nu))
    Qh = np.zeros((n + 1, sp.nx, sp.nx))
    Rh = np.zeros((n, sp.nu, sp.nu))
    Sh = np.zeros((n, sp.nu, sp.nx))
    for i, k in enumerate(ks):
        Qx, Qu, Qxu, Qux = sls.cost_blocks(sp, k, j)
        Qh[i], Rh[i], Sh[i] = Qx, Qu, Qux
    Qh[n] = sls.cost_blocks(sp, N, j)[0]
    x0 = sp.E[j][:, col]
    return A, B, Qh, Rh, Sh, x0


@pytest.mark.parametrize("tau_mode", ["zero", "uniform"])
def test_phi_columns_are_lqr_trajectories(tau_mode):
    """Each column of (Phi_x_{.,j}, Phi_u_{.,j}) is the dense-KKT LQR
    trajectory from E_j e_col under the costs Q_{.,j}."""
    sp = W.sls_small(0, tau_mode=tau_mode)
    Phix, Phiu, h, hf, _ = sls.solve(sp)
    for j in range(sp.N):
        for col in range(sp.nx):
            A, B, Qh, Rh, Sh, x0 = _column_problem(sp, j, col)
            n = A.shape[0]
            x, u, _ = lq.dense_kkt_lq(A, B, np.zeros((n, sp.nx)), Qh, Rh, Sh,
                                      np.zeros((n + 1, sp.nx)), np.zeros((n, sp.nu)), x0)
            for i in range(n + 1):
                k = j + 1 + i
                assert np.allclose(sls.block_x(sp, Phix, k, j)[:, col], x[i], atol=1e-10)
                if i < n:
                    assert np.allclose(sls.block_u(sp, Phiu, k, j)[:, col], u[i], atol=1e-10)


def test_causality_and_initial_block():
    sp = W.sls_small(1)
    Phix, Phiu, *_ = sls.solve(sp)
    for j in range(sp.N):
        assert np.allclose(sls.block_x(sp, Phix, j + 1, j), sp.E[j])
        for k in range(1, j + 1):
            assert np.all(sls.block_x(sp, Phix, k, j) == 0)
        for k in range(0, j + 1):
            assert np.all(sls.block_u(sp, Phiu, k, j) == 0)
        for k in range(j + 1, sp.N):
            nxt = sp.A[k] @ sls.block_x(sp, Phix, k, j) + sp.B[k] @ sls.block_u(sp, Phiu, k, j)
            assert np.allclose(sls.block_x(sp, Phix, k + 1, j), nxt, atol=1e-12)


def test_tau_zero_shares_gains():
    """tau = 0: the costs do not depend on j, so every j uses the same gains."""
    sp = W.sls_small(2, tau_mode="zero")
    _, _, _, _, gains = sls.solve(sp)
    for k in range(2, sp.N):
        for j in range(1, k):
            assert np.allclose(gains[(k, j)], gains[(k, 0)], atol=1e-12)


def _closed_loop_deviation(sp, Phiu, w):
    """Deviation e_k = x_k - z_k of the LTV closed loop under the
    disturbance-feedback controller, simulated through the dynamics
    e_{k+1} = A_k e_k + B_k du_k + E_k w_k with du_k = sum_{j<k} Phi_u_{k,j} w_j."""
    N, nx, nu = sp.N, sp.nx, sp.nu
    e = np.zeros((N + 1, nx))
    du = np.zeros((N, nu))
    for k in range(N):
        du[k] = sum((sls.block_u(sp, Phiu, k, j) @ w[j] for j in range(k)), np.zeros(nu))
        e[k + 1] = sp.A[k] @ e[k] + sp.B[k] @ du[k] + sp.E[k] @ w[k]
    return e, du


def test_margins_bound_monte_carlo_and_are_attained():
    """h_k bounds the constraint deviation for every unit-ball disturbance
    sequence and is attained by the adversarial one w_j = v_j / ||v_j||
    (Sec. III-A: w_k in the unit ball)."""
    sp = W.sls_small(3)
    Phix, Phiu, h, hf, _ = sls.solve(sp)
    g = np.random.default_rng(0)
    N = sp.N
    for _ in range(200):
        w = g.standard_normal((N, sp.nx))
        w /= np.maximum(1.0, np.linalg.norm(w, axis=1, keepdims=True) / g.uniform(0, 1, (N, 1)))
        e, du = _closed_loop_deviation(sp, Phiu, w)
        for k in range(N):
            dev = np.abs(sp.C[k] @ e[k] + sp.D[k] @ du[k])
            assert np.all(dev <= h[k] + 1e-12)
        assert np.all(np.abs(sp.CN @ e[N]) <= hf + 1e-12)
    for k in range(1, N):
        for c in range(sp.nc):
            w = np.zeros((N, sp.nx))
            for j in range(k):
                v = (sp.C[k] @ sls.block_x(sp, Phix, k, j) + sp.D[k] @ sls.block_u(sp, Phiu, k, j))[c]
                nv = np.linalg.norm(v)
                if nv > 0:
                    w[j] = v / nv
            e, du = _closed_loop_deviation(sp, Phiu, w)
            assert abs((sp.C[k] @ e[k] + sp.D[k] @ du[k])[c] - h[k, c]) < 1e-10


def test_state_response_matches_dynamics():
    """Phi_x from the recursion equals the simulated response to unit impulses."""
    sp = W.sls_small(4)
    Phix, Phiu, *_ = sls.solve(sp)
    g = np.random.default_rng(1)
    w = g.standard_normal((sp.N, sp.nx))
    e, _ = _closed_loop_deviation(sp, Phiu, w)
    for k in range(1, sp.N + 1):
        pred = sum(sls.block_x(sp, Phix, k, j) @ w[j] for j in range(k))
        assert np.allclose(e[k], pred, atol=1e-12)


@pytest.mark.parametrize("tau_mode", ["zero", "uniform"])
def test_scan_form_reproduces_sls_riccati(tau_mode):
    """The SLS scan of Sec. IV-B (eq. robust_combin, the homogeneous version of
    eq. combination_rules) with leaves A~ = A - B Qu^{-1} Qux,
    D~ = B Qu^{-1} B^T, P~ = Qx - Qxu Qu^{-1} Qux and terminal (Qx_N, 0, 0)
    gives P_k^{(j)} = P~_{k,N+1}."""
    sp = W.sls_small(5, tau_mode=tau_mode)
    N = sp.N
    for j in range(N):
        _, Pj = sls.riccati_j(sp, j)
        els = []
        for k in range(j + 1, N):
            Qx, Qu, Qxu, Qux = sls.cost_blocks(sp, k, j)
            Qi = np.linalg.inv(Qu)
            els.append(scan.Elem(P=Qx - Qxu @ Qi @ Qux, p=np.zeros(sp.nx), A=sp.A[k] - sp.B[k] @ Qi @ Qux,
                                 C=sp.B[k] @ Qi @ sp.B[k].T, b=np.zeros(sp.nx)))
        els.append(scan.Elem(P=sls.cost_blocks(sp, N, j)[0], p=np.zeros(sp.nx), A=np.zeros((sp.nx, sp.nx)),
                             C=np.zeros((sp.nx, sp.nx)), b=np.zeros(sp.nx)))
        s = scan.suffix_scan(els)
        for i, k in enumerate(range(j + 1, N + 1)):
            assert np.allclose(s[i].P, Pj[k], atol=1e-10)


def test_beta_tau_definition():
    sp = W.sls_small(6)
    Phix, Phiu, *_ = sls.solve(sp)
    lam = np.zeros((sp.N, sp.nc))
    lam_t = np.zeros(sp.nf)
    assert np.all(sls.beta_tau(sp, Phix, Phiu, lam, lam_t) == 0)
    g = np.random.default_rng(0)
    lam = np.abs(g.standard_normal((sp.N, sp.nc)))
    lam_t = np.abs(g.standard_normal(sp.nf))
    t1 = sls.beta_tau(sp, Phix, Phiu, lam, lam_t)
    t2 = sls.beta_tau(sp, Phix, Phiu, 2 * lam, 2 * lam_t)
    assert np.allclose(t2, 2 * t1)
    k, j = sp.N - 1, 0
    M = sp.C[k] @ sls.block_x(sp, Phix, k, j) + sp.D[k] @ sls.block_u(sp, Phiu, k, j)
    assert np.allclose(t1[k, j, :sp.nc], lam[k] / np.sqrt(np.sum(M ** 2, axis=1) + 1e-8))
