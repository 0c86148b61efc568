"""FP64 KKT residual of the LTV-QP eq. sqp_qp.

Test infrastructure only (see oracle/__init__.py).

The paper leaves "residual" undefined (Sec. V-A uses a maximum residual
tolerance).  Reading: absolute infinity-norm KKT residual, the max of
  (i)   dynamics and initial-state residual,
  (ii)  bound violation max(G xi - hi, lo - G xi, 0),
  (iii) stationarity in u after recovering the costate mu by the backward pass
        mu_N = Q_N x_N + q_N + C_N^T lam_N,
        mu_k = Q_k x_k + S_k^T u_k + q_k + C_k^T lam_k + A_k^T mu_{k+1},
        residual R_k u_k + S_k x_k + r_k + D_k^T lam_k + B_k^T mu_{k+1},
  (iv)  complementarity |lam_i| * slack_i, slack measured to the bound the sign
        of lam_i points at (lam_i > 0: upper, lam_i < 0: lower); a multiplier
        pointing at an infinite bound counts |lam_i| in full.
The Lagrangian sign convention is that of eq. lagrangian.
"""
from __future__ import annotations

import numpy as np

from .lq import G_apply, stage_rows


def kkt_parts(qp, x, u, lam) -> dict:
    N = qp.N
    dyn = np.max(np.abs(x[0] - qp.x0)) if qp.nx else 0.0
    for k in range(N):
        dyn = max(dyn, np.max(np.abs(x[k + 1] - qp.A[k] @ x[k] - qp.B[k] @ u[k] - qp.c[k])))
    v = G_apply(qp, x, u)
    viol = 0.0
    if qp.m:
        viol = float(np.max(np.maximum(np.maximum(v - qp.hi, qp.lo - v), 0.0)))
    mu = qp.Q[N] @ x[N] + qp.q[N] + qp.CN.T @ stage_rows(qp, lam, N)
    stat = 0.0
    for k in range(N - 1, -1, -1):
        lk = stage_rows(qp, lam, k)
        ru = qp.R[k] @ u[k] + qp.S[k] @ x[k] + qp.r[k] + qp.D[k].T @ lk + qp.B[k].T @ mu
        stat = max(stat, float(np.max(np.abs(ru))) if qp.nu else 0.0)
        mu = qp.Q[k] @ x[k] + qp.S[k].T @ u[k] + qp.q[k] + qp.C[k].T @ lk + qp.A[k].T @ mu
    comp = 0.0
    for i in range(qp.m):
        li = lam[i]
        if li > 0:
            c = li * abs(qp.hi[i] - v[i]) if np.isfinite(qp.hi[i]) else abs(li)
        elif li < 0:
            c = -li * abs(v[i] - qp.lo[i]) if np.isfinite(qp.lo[i]) else abs(li)
        else:
            c = 0.0
        comp = max(comp, c)
    return dict(dyn=float(dyn), viol=viol, stat=stat, comp=float(comp))


def kkt_residual(qp, x, u, lam) -> float:
    p = kkt_parts(qp, x, u, lam)
    return max(p.values())


def u_residuals(qp, x, u, lam) -> np.ndarray:
    """Per-stage u-stationarity residuals R_k u_k + S_k x_k + r_k + D_k^T lam_k
    + B_k^T mu_{k+1} with the costate of kkt_parts (the part of the KKT residual
    that iterative refinement feeds back), shape [N, nu]."""
    N = qp.N
    out = np.zeros((N, qp.nu))
    mu = qp.Q[N] @ x[N] + qp.q[N] + qp.CN.T @ stage_rows(qp, lam, N)
    for k in range(N - 1, -1, -1):
        lk = stage_rows(qp, lam, k)
        out[k] = qp.R[k] @ u[k] + qp.S[k] @ x[k] + qp.r[k] + qp.D[k].T @ lk + qp.B[k].T @ mu
        mu = qp.Q[k] @ x[k] + qp.S[k].T @ u[k] + qp.q[k] + qp.C[k].T @ lk + qp.A[k].T @ mu
    return out
