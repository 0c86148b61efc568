"""Primal infeasibility certificate of the LTV-QP (eq. sqp_qp) from a
multiplier direction, by Farkas' lemma.

Test infrastructure only (see oracle/__init__.py).

The constraints of the QP in xi = (x_0 .. x_N, u_0 .. u_{N-1}) are
  E xi = e:  x_0 = x0 and x_{k+1} - A_k x_k - B_k u_k = c_k (k < N),
  lo <= G xi <= hi:  rows C_k x_k + D_k u_k (k < N) and C_N x_N.
For any feasible xi and any (mu, w) with E^T mu + G^T w = 0,
  0 = w^T G xi + mu^T E xi <= sigma(w) + e^T mu,
sigma(w) = sum_i (w_i > 0 ? hi_i w_i : lo_i w_i) the support function of the
box, so sigma(w) + e^T mu < 0 proves that no feasible xi exists.  Given w,
the x-components of E^T mu + G^T w = 0 determine mu (nu_k the multiplier of
the dynamics row of stage k, mu_0 that of x_0 = x0):
  x_N:  nu_{N-1} + C_N^T w_N = 0,
  x_k:  nu_{k-1} - A_k^T nu_k + C_k^T w_k = 0   (1 <= k <= N-1),
  x_0:  mu_0 - A_0^T nu_0 + C_0^T w_0 = 0,
and the u-components leave the residual r_k = D_k^T w_k - B_k^T nu_k.

Reading (the paper has no infeasibility detection; this is the library's
classification of a solve that reached its iteration limit, in the manner of
OSQP's certificate): w is the change of the unscaled multipliers lambda =
rho y over the last check interval before the limit; with W = ||w||_inf > 0
the certificate holds when every w_i that pushes against an infinite bound is
at most tol W, ||r||_inf <= tol W and sigma(w) + e^T mu < -tol W.
"""
from __future__ import annotations

import numpy as np


def multipliers(qp, w):
    """(nu [N, nx], mu0 [nx], r [N, nu]) of the recursion in the module
    docstring for the row multipliers w [N nc + nf]."""
    N, nx, nu, nc, nf = qp.N, qp.nx, qp.nu, qp.nc, qp.nf
    w = np.asarray(w, dtype=float)
    wk = w[:N * nc].reshape(N, nc)
    wN = w[N * nc:]
    nu_ = np.zeros((N, nx))
    nu_[N - 1] = -(qp.CN.T @ wN) if nf else 0.0
    for k in range(N - 1, 0, -1):
        nu_[k - 1] = qp.A[k].T @ nu_[k] - qp.C[k].T @ wk[k]
    mu0 = qp.A[0].T @ nu_[0] - qp.C[0].T @ wk[0]
    r = np.stack([qp.D[k].T @ wk[k] - qp.B[k].T @ nu_[k] for k in range(N)])
    return nu_, mu0, r


def support(qp, w, W):
    """sigma(w) over the finite bounds, and the largest |w_i| that pushes
    against an infinite bound (w_i > 0 with hi_i = inf, w_i < 0 with
    lo_i = -inf)."""
    sig, push = 0.0, 0.0
    for wi, lo, hi in zip(np.asarray(w, dtype=float), qp.lo, qp.hi):
        if wi > 0.0:
            if np.isfinite(hi):
                sig += hi * wi
            else:
                push = max(push, wi)
        elif wi < 0.0:
            if np.isfinite(lo):
                sig += lo * wi
            else:
                push = max(push, -wi)
    return sig, push


def certificate(qp, w, tol: float) -> dict:
    """The certificate test of the module docstring for direction w."""
    w = np.asarray(w, dtype=float)
    W = float(np.max(np.abs(w))) if w.size else 0.0
    nu_, mu0, r = multipliers(qp, w)
    sig, push = support(qp, w, W)
    value = sig + float(qp.x0 @ mu0) + float(np.sum(qp.c * nu_))
    r_max = float(np.max(np.abs(r))) if r.size else 0.0
    certified = W > 0.0 and push <= tol * W and r_max <= tol * W and value < -tol * W
    return dict(certified=bool(certified), value=value, r_max=r_max, W=W, push=push, nu=nu_, mu0=mu0, r=r)
