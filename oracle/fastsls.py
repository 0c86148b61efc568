"""The FastSLS alternation between the tightened nominal QP and the robust
controller (Sec. III-D, eq. nmpc_problem_tightened, eq. fastsls_qp, App. B,
Fig. fig:schematic).

Test infrastructure only (see oracle/__init__.py).

One step of the alternation, given the duals tau of the previous step
(tau = None on the first step: the controller problem without constraint
weights, eq. fastsls_qp with tau = 0):
  1. controller update: the SLS solve with the cost blocks of
     eq. sls_cost_matrices_tau -> Phi_x, Phi_u and the margins h_k, h^f;
  2. tightening: the nominal constraints g + h <= 0 of
     eq. nmpc_problem_tightened, i.e. the bounds of the LTV-QP moved inwards
     by the margins;
  3. nominal update: the tightened LTV-QP solved exactly (oracle.admm.
     exact_solution), giving (dx, du) and the unscaled multipliers lambda;
  4. duals: tau_{k,j} = lambda_k / sqrt(beta_{k,j} + eps) (App. B) from the
     new lambda and the Phi of step 1.
This is the order of the RTI variant of Sec. IV-C (the controller update
warm-started from the previous tau, then the tightened nominal solve); the
nominal trajectory returned by a step is feasible for the tightening of the
same step.

Readings:
  * two-sided rows lo <= G xi <= hi are two one-sided rows of the paper's
    g <= 0 form with the same row vector up to sign; the disturbance moves
    both by the same row norm, so both bounds are tightened by h:
    lo + h <= G xi <= hi - h.  At most one of the two is active, with
    multiplier |lambda| (lambda > 0 at the upper bound, < 0 at the lower), so
    tau uses |lambda|.
  * h_0 = 0 (no disturbance acts before stage 1), so stage-0 rows keep their
    bounds.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import sls
from .admm import exact_solution


def tighten(qp, h, hf):
    """Bounds of eq. nmpc_problem_tightened: stage-k rows lo + h_k, hi - h_k,
    terminal rows lo + h^f, hi - h^f (infinite bounds stay infinite)."""
    m = np.concatenate([np.asarray(h, dtype=float).reshape(-1), np.asarray(hf, dtype=float).reshape(-1)])
    return dataclasses.replace(qp, lo=qp.lo + m, hi=qp.hi - m)


def taus(sp, Phix, Phiu, lam, eps: float = 1e-8):
    """App. B duals from the unscaled QP multipliers lam [N nc + nf] with the
    |lambda| reading for two-sided rows."""
    N, nc = sp.N, sp.nc
    lam = np.abs(np.asarray(lam, dtype=float))
    return sls.beta_tau(sp, Phix, Phiu, lam[:N * nc].reshape(N, nc), lam[N * nc:], eps)


def step(qp, sp, tau=None, eps: float = 1e-8, qp_solver=exact_solution):
    """One alternation step (module docstring); returns a dict with Phix,
    Phiu, h, hf, the tightened QP, x, u, lam and the new tau."""
    Phix, Phiu, h, hf, _ = sls.solve(dataclasses.replace(sp, tau=tau))
    qt = tighten(qp, h, hf)
    x, u, lam = qp_solver(qt)
    return dict(Phix=Phix, Phiu=Phiu, h=h, hf=hf, qp=qt, x=x, u=u, lam=lam, tau=taus(sp, Phix, Phiu, lam, eps))


def alternation(qp, sp, iters: int, tau0=None, eps: float = 1e-8, qp_solver=exact_solution):
    """`iters` alternation steps from tau0 (None: zero); the list of steps."""
    out = []
    tau = tau0
    for _ in range(iters):
        s = step(qp, sp, tau, eps, qp_solver)
        out.append(s)
        tau = s["tau"]
    return out
