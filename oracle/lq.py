"""LQ pieces of the ADMM primal update (Sec. IV-A, eq. primal_update).

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


def stage_rows(qp, v: np.ndarray, k: int) -> np.ndarray:
    """Slice of a constraint-space vector belonging to stage k (k == N: terminal)."""
    nc, N = qp.nc, qp.N
    if k < N:
        return v[k * nc:(k + 1) * nc]
    return v[N * nc:]


def augmented(qp, rho: float):
    """Augmented cost matrices, eq. augmented_matrices (Sec. IV-A).

    Q^_k = Q_k + rho C_k^T C_k,  R^_k = R_k + rho D_k^T D_k,
    S^_k = S_k + rho D_k^T C_k   (reading: the printed rho C^T D is nx-by-nu but
    S_k is nu-by-nx, so the transposed product D^T C is meant),
    Q^_N = Q_N + rho C_N^T C_N.
    """
    N = qp.N
    Qh = np.empty_like(qp.Q)
    Rh = np.empty_like(qp.R)
    Sh = np.empty_like(qp.S)
    for k in range(N):
        Qh[k] = qp.Q[k] + rho * qp.C[k].T @ qp.C[k]
        Rh[k] = qp.R[k] + rho * qp.D[k].T @ qp.D[k]
        Sh[k] = qp.S[k] + rho * qp.D[k].T @ qp.C[k]
    Qh[N] = qp.Q[N] + rho * qp.CN.T @ qp.CN
    return Qh, Rh, Sh


def augmented_linear(qp, rho: float, y: np.ndarray, z: np.ndarray):
    """Augmented linear terms with the scaled dual y = lambda / rho,
    eq. augmented_linear: q^_k = q_k + rho C_k^T (y_k - z_k),
    r^_k = r_k + rho D_k^T (y_k - z_k), q^_N = q_N + rho C_N^T (y_N - z_N)."""
    N = qp.N
    w = y - z
    qh = np.empty_like(qp.q)
    rh = np.empty_like(qp.r)
    for k in range(N):
        wk = stage_rows(qp, w, k)
        qh[k] = qp.q[k] + rho * qp.C[k].T @ wk
        rh[k] = qp.r[k] + rho * qp.D[k].T @ wk
    qh[N] = qp.q[N] + rho * qp.CN.T @ stage_rows(qp, w, N)
    return qh, rh


def riccati(A, B, c, Qh, Rh, Sh, qh, rh):
    """Sequential Riccati recursion for the LQ problem eq. primal_update, the
    textbook form behind eq. controller_cache (Sec. IV-A.1):

        P_N = Q^_N, p_N = q^_N, and for k = N-1 .. 0
        Gamma_k = (R^_k + B_k^T P_{k+1} B_k)^{-1}
        K_k = -Gamma_k (S^_k + B_k^T P_{k+1} A_k)
        k_k = -Gamma_k (B_k^T (p_{k+1} + P_{k+1} b_k) + r^_k)
        P_k = Q^_k + A_k^T P_{k+1} A_k + (S^_k + B_k^T P_{k+1} A_k)^T K_k
        p_k = q^_k + S^_k^T k_k + A_k^T (p_{k+1} + P_{k+1} (B_k k_k + b_k))

    Returns P [N+1], p [N+1], K [N], kff [N], Gamma [N].
    """
    N, nx = A.shape[0], A.shape[1]
    nu = B.shape[2]
    P = np.zeros((N + 1, nx, nx))
    p = np.zeros((N + 1, nx))
    K = np.zeros((N, nu, nx))
    kff = np.zeros((N, nu))
    Gam = np.zeros((N, nu, nu))
    P[N] = Qh[N]
    p[N] = qh[N]
    for k in range(N - 1, -1, -1):
        Pn, pn = P[k + 1], p[k + 1]
        G = np.linalg.inv(Rh[k] + B[k].T @ Pn @ B[k])
        Bx = Sh[k] + B[k].T @ Pn @ A[k]
        K[k] = -G @ Bx
        kff[k] = -G @ (B[k].T @ (pn + Pn @ c[k]) + rh[k])
        P[k] = Qh[k] + A[k].T @ Pn @ A[k] + Bx.T @ K[k]
        p[k] = qh[k] + Sh[k].T @ kff[k] + A[k].T @ (pn + Pn @ (B[k] @ kff[k] + c[k]))
        Gam[k] = G
    return P, p, K, kff, Gam


def rollout(A, B, c, K, kff, x0):
    """Forward pass dx_{k+1} = A_k dx_k + B_k du_k + b_k with du_k = K_k dx_k + k_k
    (eq. nom_recovery written sequentially)."""
    N, nx = A.shape[0], A.shape[1]
    nu = B.shape[2]
    x = np.zeros((N + 1, nx))
    u = np.zeros((N, nu))
    x[0] = x0
    for k in range(N):
        u[k] = K[k] @ x[k] + kff[k]
        x[k + 1] = A[k] @ x[k] + B[k] @ u[k] + c[k]
    return x, u


def lq_solve(qp, Qh, Rh, Sh, qh, rh, x0):
    """Solve eq. primal_update by the sequential Riccati recursion."""
    P, p, K, kff, _ = riccati(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh)
    return rollout(qp.A, qp.B, qp.c, K, kff, x0)


def dense_kkt_lq(A, B, c, Qh, Rh, Sh, qh, rh, x0, extra_eq=None):
    """Solve the equality-constrained QP eq. primal_update as one dense KKT
    system (independent of the Riccati recursion; used as a pin).

    Variables xi = (x_0..x_N, u_0..u_{N-1}).  extra_eq = (E, e) appends extra
    equality rows E xi = e (used by the active-set brute force).
    Returns x [N+1, nx], u [N, nu], and the multipliers of all equality rows.
    """
    N, nx = A.shape[0], A.shape[1]
    nu = B.shape[2]
    nX = (N + 1) * nx
    n = nX + N * nu
    H = np.zeros((n, n))
    g = np.zeros(n)

    def xi(k):
        return slice(k * nx, (k + 1) * nx)

    def ui(k):
        return slice(nX + k * nu, nX + (k + 1) * nu)

    for k in range(N):
        H[xi(k), xi(k)] += Qh[k]
        H[ui(k), ui(k)] += Rh[k]
        H[ui(k), xi(k)] += Sh[k]
        H[xi(k), ui(k)] += Sh[k].T
        g[xi(k)] += qh[k]
        g[ui(k)] += rh[k]
    H[xi(N), xi(N)] += Qh[N]
    g[xi(N)] += qh[N]
    rows = []
    rhs = []
    E0 = np.zeros((nx, n))
    E0[:, xi(0)] = np.eye(nx)
    rows.append(E0)
    rhs.append(x0)
    for k in range(N):
        Ek = np.zeros((nx, n))
        Ek[:, xi(k + 1)] = np.eye(nx)
        Ek[:, xi(k)] = -A[k]
        Ek[:, ui(k)] = -B[k]
        rows.append(Ek)
        rhs.append(c[k])
    if extra_eq is not None and extra_eq[0].shape[0]:
        rows.append(extra_eq[0])
        rhs.append(extra_eq[1])
    E = np.vstack(rows)
    e = np.concatenate(rhs)
    m = E.shape[0]
    KKT = np.zeros((n + m, n + m))
    KKT[:n, :n] = H
    KKT[:n, n:] = E.T
    KKT[n:, :n] = E
    sol = np.linalg.solve(KKT, np.concatenate([-g, e]))
    xi_ = sol[:n]
    x = xi_[:nX].reshape(N + 1, nx)
    u = xi_[nX:].reshape(N, nu)
    return x, u, sol[n:]


def G_apply(qp, x, u) -> np.ndarray:
    """G(dx, du) = (C_k dx_k + D_k du_k for k < N; C_N dx_N), Sec. IV-A."""
    N = qp.N
    out = np.empty(qp.m)
    for k in range(N):
        out[k * qp.nc:(k + 1) * qp.nc] = qp.C[k] @ x[k] + qp.D[k] @ u[k]
    out[N * qp.nc:] = qp.CN @ x[N]
    return out


def GT_apply(qp, w: np.ndarray):
    """Adjoint G^T w = (C_k^T w_k, D_k^T w_k; C_N^T w_N)."""
    N = qp.N
    gx = np.zeros((N + 1, qp.nx))
    gu = np.zeros((N, qp.nu))
    for k in range(N):
        wk = stage_rows(qp, w, k)
        gx[k] = qp.C[k].T @ wk
        gu[k] = qp.D[k].T @ wk
    gx[N] = qp.CN.T @ stage_rows(qp, w, N)
    return gx, gu


def H_apply(qp, x, u):
    """Block-diagonal Hessian of J_QP applied to (x, u): (Q x + S^T u, R u + S x;
    Q_N x_N)."""
    N = qp.N
    hx = np.zeros((N + 1, qp.nx))
    hu = np.zeros((N, qp.nu))
    for k in range(N):
        hx[k] = qp.Q[k] @ x[k] + qp.S[k].T @ u[k]
        hu[k] = qp.R[k] @ u[k] + qp.S[k] @ x[k]
    hx[N] = qp.Q[N] @ x[N]
    return hx, hu


def objective(qp, x, u) -> float:
    """J_QP of eq. sqp_qp."""
    J = 0.0
    for k in range(qp.N):
        J += 0.5 * x[k] @ qp.Q[k] @ x[k] + u[k] @ qp.S[k] @ x[k] + 0.5 * u[k] @ qp.R[k] @ u[k]
        J += qp.q[k] @ x[k] + qp.r[k] @ u[k]
    J += 0.5 * x[qp.N] @ qp.Q[qp.N] @ x[qp.N] + qp.q[qp.N] @ x[qp.N]
    return float(J)
