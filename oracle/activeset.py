"""Active-set solves of the LTV-QP eq. sqp_qp by dense KKT systems.

Test infrastructure only (see oracle/__init__.py).

brute_force() enumerates every assignment of each finite bound row to
{inactive, at lower bound, at upper bound}, solves the equality-constrained
QP with the active rows as equalities (dense KKT), and keeps a point that
satisfies primal feasibility and dual sign conditions.  Q, R > 0 make the
minimiser unique, so any accepted active set gives the same primal point.
"""
from __future__ import annotations

import itertools

import numpy as np

from .lq import G_apply, dense_kkt_lq


def _G_rows(qp):
    """Dense matrix of G acting on xi = (x_0..x_N, u_0..u_{N-1})."""
    N, nx, nu, nc = qp.N, qp.nx, qp.nu, qp.nc
    nX = (N + 1) * nx
    n = nX + N * nu
    Gm = np.zeros((qp.m, n))
    for k in range(N):
        Gm[k * nc:(k + 1) * nc, k * nx:(k + 1) * nx] = qp.C[k]
        Gm[k * nc:(k + 1) * nc, nX + k * nu:nX + (k + 1) * nu] = qp.D[k]
    Gm[N * nc:, N * nx:(N + 1) * nx] = qp.CN
    return Gm


def solve_active(qp, active: dict):
    """Equality-constrained solve with rows active[i] in {'lo', 'hi'} pinned.
    Returns x, u, lam (lam_i > 0 at upper, < 0 at lower bound)."""
    Gm = _G_rows(qp)
    idx = sorted(active)
    E = Gm[idx] if idx else np.zeros((0, Gm.shape[1]))
    e = np.array([qp.hi[i] if active[i] == "hi" else qp.lo[i] for i in idx])
    x, u, mult = dense_kkt_lq(qp.A, qp.B, qp.c, qp.Q, qp.R, qp.S, qp.q, qp.r, qp.x0, extra_eq=(E, e))
    n_dyn = (qp.N + 1) * qp.nx
    lam = np.zeros(qp.m)
    for j, i in enumerate(idx):
        lam[i] = mult[n_dyn + j]
    return x, u, lam


def brute_force(qp, tol: float = 1e-9):
    rows = list(range(qp.m))
    choices = []
    for i in rows:
        c = [None]
        if np.isfinite(qp.lo[i]):
            c.append("lo")
        if np.isfinite(qp.hi[i]):
            c.append("hi")
        choices.append(c)
    best = None
    for combo in itertools.product(*choices):
        act = {i: c for i, c in zip(rows, combo) if c is not None}
        try:
            x, u, lam = solve_active(qp, act)
        except np.linalg.LinAlgError:
            continue
        v = G_apply(qp, x, u)
        if np.any(v > qp.hi + tol) or np.any(v < qp.lo - tol):
            continue
        ok = True
        for i, c in act.items():
            if c == "hi" and lam[i] < -tol:
                ok = False
            if c == "lo" and lam[i] > tol:
                ok = False
        if ok:
            best = (x, u, lam, act)
            break
    if best is None:
        raise RuntimeError("no KKT point found (infeasible instance?)")
    return best


def polish(qp, x, u, lam, tol: float = 1e-7):
    """Dense-KKT solve on the active set detected from an approximate
    solution: rows whose multiplier is nonzero or whose value sits at a bound."""
    v = G_apply(qp, x, u)
    act = {}
    scale = max(1.0, float(np.max(np.abs(lam))) if lam.size else 1.0)
    for i in range(qp.m):
        if lam[i] > tol * scale and np.isfinite(qp.hi[i]):
            act[i] = "hi"
        elif lam[i] < -tol * scale and np.isfinite(qp.lo[i]):
            act[i] = "lo"
    xs, us, ls = solve_active(qp, act)
    return xs, us, ls
