"""SLS controller synthesis and reachability margins (Sec. III-D, Sec. IV-B,
App. B).

Test infrastructure only (see oracle/__init__.py).

The problem eq. fastsls_qp decouples over the disturbance index j into N
independent LQR problems in the matrix variables Phi_{k,j}; the oracle solves
them with the N Riccati recursions eq. backward_prop and the forward
propagation eq. forward_prop, written as plain loops.

Readings:
  * Phi_{k,j} = 0 for k <= j (strict causality, eq. disturbance_feedback);
    the "k = j" terms of the cost therefore vanish.
  * the terminal cost block is Qx_{N,j} (the printed Qx_{N+1} is a typo).
  * the scan leaves of Sec. IV-B are written with Q^{xu}; for the dimensions to
    match they must use the transposed block Q^{ux} in A~ = A - B Qu^{-1} Qux
    and Q^{xu} Qu^{-1} Q^{ux} in P~ (as in the QP leaves of eq. assoc_init).
  * tau layout [N+1, N, max(nc, nf)]: tau[k, j, :nc] for stage k < N and
    tau[N, j, :nf] for the terminal rows; tau = None means zero.
"""
from __future__ import annotations

import numpy as np


def cost_blocks(sp, k: int, j: int):
    """eq. sls_cost_matrices_tau: Q^T Q with Q = (diag(sqrt tau) [C D],
    blkdiag(Qbar^1/2, Rbar^1/2)) gives
    Qx = Qbar + C^T diag(tau) C, Qu = Rbar + D^T diag(tau) D,
    Qxu = C^T diag(tau) D, Qux = Qxu^T; terminal Qx_N = QbarN + C_N^T diag(tau) C_N."""
    if k < sp.N:
        t = np.zeros(sp.nc) if sp.tau is None else sp.tau[k, j, :sp.nc]
        Ct, Dt = sp.C[k], sp.D[k]
        Qx = sp.Qbar + Ct.T @ (t[:, None] * Ct)
        Qu = sp.Rbar + Dt.T @ (t[:, None] * Dt)
        Qxu = Ct.T @ (t[:, None] * Dt)
        return Qx, Qu, Qxu, Qxu.T
    t = np.zeros(sp.nf) if sp.tau is None else sp.tau[sp.N, j, :sp.nf]
    return sp.QbarN + sp.CN.T @ (t[:, None] * sp.CN), None, None, None


def riccati_j(sp, j: int):
    """eq. backward_prop for disturbance index j: P_N = Qx_{N,j}; for
    k = N-1 .. j+1: Gk = (Qu + B^T P B)^{-1}, Bk = Qux + B^T P A, Kk = -Gk Bk,
    Pk = Qx + A^T P A + Kk^T Bk.  Returns {k: K_k^{(j)}} and {k: P_k^{(j)}}."""
    N = sp.N
    P = {N: cost_blocks(sp, N, j)[0]}
    K = {}
    for k in range(N - 1, j, -1):
        Qx, Qu, Qxu, Qux = cost_blocks(sp, k, j)
        Pn = P[k + 1]
        G = np.linalg.inv(Qu + sp.B[k].T @ Pn @ sp.B[k])
        Bk = Qux + sp.B[k].T @ Pn @ sp.A[k]
        K[k] = -G @ Bk
        P[k] = Qx + sp.A[k].T @ Pn @ sp.A[k] + K[k].T @ Bk
    return K, P


def solve(sp):
    """Phi_x [N*nx, N*nx] (block row k-1 holds Phi_x_{k,.} for k = 1..N, block
    column j), Phi_u [N*nu, N*nx] (block row k for k = 0..N-1), margins
    h [N, nc], hf [nf] (the stacked constraint tightenings of Sec. III-D) and
    the gains {(k, j): K}."""
    N, nx, nu = sp.N, sp.nx, sp.nu
    Phix = np.zeros((N * nx, N * nx))
    Phiu = np.zeros((N * nu, N * nx))
    gains = {}
    for j in range(N):
        K, _ = riccati_j(sp, j)
        X = sp.E[j].copy()                      # Phi_x_{j+1, j} = E_j
        for k in range(j + 1, N + 1):
            Phix[(k - 1) * nx:k * nx, j * nx:(j + 1) * nx] = X
            if k == N:
                break
            U = K[k] @ X                         # Phi_u_{k, j} = K_k^{(j)} Phi_x_{k, j}
            Phiu[k * nu:(k + 1) * nu, j * nx:(j + 1) * nx] = U
            gains[(k, j)] = K[k]
            X = (sp.A[k] + sp.B[k] @ K[k]) @ X
    h, hf = margins(sp, Phix, Phiu)
    return Phix, Phiu, h, hf, gains


def block_x(sp, Phix, k, j):
    nx = sp.nx
    return Phix[(k - 1) * nx:k * nx, j * nx:(j + 1) * nx]


def block_u(sp, Phiu, k, j):
    nx, nu = sp.nx, sp.nu
    return Phiu[k * nu:(k + 1) * nu, j * nx:(j + 1) * nx]


def margins(sp, Phix, Phiu):
    """Constraint tightenings (Sec. III-D):
    h_k = sum_{j<k} || C_k Phi_x_{k,j} + D_k Phi_u_{k,j} ||_{2,row},
    h^f = sum_{j<N} || C_N Phi_x_{N,j} ||_{2,row}."""
    N = sp.N
    h = np.zeros((N, sp.nc))
    for k in range(1, N):
        for j in range(k):
            M = sp.C[k] @ block_x(sp, Phix, k, j) + sp.D[k] @ block_u(sp, Phiu, k, j)
            h[k] += np.linalg.norm(M, axis=1)
    hf = np.zeros(sp.nf)
    for j in range(N):
        hf += np.linalg.norm(sp.CN @ block_x(sp, Phix, N, j), axis=1)
    return h, hf


def beta_tau(sp, Phix, Phiu, lam_stage, lam_term, eps: float = 1e-8):
    """App. B: beta_{k,j} = ||C_k Phi_x_{k,j} + D_k Phi_u_{k,j}||^2_{2,row}
    (elementwise square), beta_{N,j} = ||C_N Phi_x_{N,j}||^2_{2,row},
    tau_{k,j} = lam_k / sqrt(beta_{k,j} + eps).  lam_stage [N, nc] and
    lam_term [nf] are the unscaled QP duals.  Returns tau in the
    [N+1, N, max(nc, nf)] layout (zero where k <= j)."""
    N = sp.N
    w = max(sp.nc, sp.nf)
    tau = np.zeros((N + 1, N, w))
    for j in range(N):
        for k in range(j + 1, N):
            M = sp.C[k] @ block_x(sp, Phix, k, j) + sp.D[k] @ block_u(sp, Phiu, k, j)
            beta = np.sum(M * M, axis=1)
            tau[k, j, :sp.nc] = lam_stage[k] / np.sqrt(beta + eps)
        M = sp.CN @ block_x(sp, Phix, N, j)
        beta = np.sum(M * M, axis=1)
        tau[N, j, :sp.nf] = lam_term / np.sqrt(beta + eps)
    return tau
