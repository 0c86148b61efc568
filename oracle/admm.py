"""Step-by-step ADMM for the LTV-QP (Sec. IV-A, eq. admm_qp .. z/lambda
updates), with the LQ subproblem solved by the sequential Riccati recursion.

Test infrastructure only (see oracle/__init__.py).

Readings (the paper is silent or garbled here):
  * constraints are two-sided, lo <= G xi <= hi with +-inf allowed; the
    projection is clamp(v + y, lo, hi), which is the printed min(v + y, f)
    when lo = -inf.
  * no over-relaxation, no proximal term.
  * cold start z = y = 0, rho0 = 0.1.
  * residuals: r_prim = ||v - z+||_inf, r_dual = ||rho G^T (z+ - z)||_inf;
    the stop test r_prim <= eps and r_dual <= eps runs every check_every
    iterations.
  * rho rule "similar to OSQP Sec. 5.2": every sigma iterations
        rho_new = rho * sqrt( (r_prim / max(||v||, ||z+||))
                             / (r_dual / max(||H xi||, ||G^T lam||, ||(q, r)||)) ),
    clamped to [rho_min, rho_max], applied only when it moves rho by more than
    5x; y is rescaled by rho_old / rho_new so that lam = rho y is continuous,
    and the cost matrices are re-augmented (the "refactor").
  * "solve to a KKT tolerance": when the in-loop test passes, the FP64 KKT
    residual (oracle.kkt) is evaluated; if it exceeds eps_kkt the in-loop
    tolerance is divided by 10, but not below eps_floor, and iterations
    continue; at the floor a failing check triggers one round of iterative
    refinement (at most max_refine rounds): the FP64 u-stationarity residual
    ru_k (oracle.kkt.u_residuals) is added to the linear term r_k used by the
    iteration (and by the rho rule's ||(q, r)||), while the KKT check keeps the
    original data.
  * stall rule (option stall_iters > 0, used to mirror FP32 solves): once the
    in-loop tolerance has sat at eps_floor for stall_iters iterations without
    the in-loop test passing, the next stop-test iteration runs the KKT check
    anyway (and refines on failure), as if the test had passed.  Rounding in a
    reduced-precision LQ solve can hold r_prim or r_dual just above the floor;
    in exact arithmetic both go to zero and the rule never fires.

  * a solve that reaches max_iter is classified by the primal infeasibility
    certificate of oracle.infeas, taken from the change of lambda = rho y
    over the last check interval (reference point saved at iteration
    max_iter - check_every).

The KKT gate, the tightening of eps, the refinement, the stall rule and the
infeasibility classification are this project's stopping rule: the paper stops ADMM on its residual tolerance
alone and prints no such control.  With eps_kkt = None (the default) the
oracle runs the paper's ADMM and stops on r_prim, r_dual <= eps.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import dataclasses

from .infeas import certificate
from .kkt import kkt_residual, u_residuals
from .lq import G_apply, GT_apply, H_apply, augmented, augmented_linear, lq_solve


@dataclass
class Settings:
    rho0: float = 0.1
    eps: float = 1e-4
    eps_kkt: float | None = None   # None: stop on the in-loop test alone
    eps_floor: float = 1e-7        # lowest in-loop tolerance the KKT gate tightens to
    max_refine: int = 3            # refinement rounds allowed at the floor
    stall_iters: int = 0           # > 0: stall rule (module docstring); 0 off
    sigma: int = 25                # 0: fixed rho
    check_every: int = 5
    max_iter: int = 4000
    rho_min: float = 1e-6
    rho_max: float = 1e6


@dataclass
class Result:
    x: np.ndarray
    u: np.ndarray
    z: np.ndarray
    y: np.ndarray
    rho: float
    lam: np.ndarray
    iters: int
    r_prim: float
    r_dual: float
    converged: bool
    refactors: int
    rho_hist: list = field(default_factory=list)
    kkt: float | None = None
    infeasible: bool = False       # reached max_iter with a primal infeasibility certificate


def residuals(qp, v, z_new, z, rho):
    """Primal and dual residuals of one iteration (Sec. IV-A):
    r_prim = ||v - z+||_inf, r_dual = ||rho G^T (z+ - z)||_inf."""
    r_prim = float(np.max(np.abs(v - z_new))) if qp.m else 0.0
    gx, gu = GT_apply(qp, rho * (z_new - z))
    r_dual = float(max(np.max(np.abs(gx)), np.max(np.abs(gu)) if gu.size else 0.0))
    return r_prim, r_dual


def rho_rule(qp, x, u, v, z_new, y_new, rho, r_prim, r_dual, s: Settings) -> float:
    """OSQP-style rho proposal (see module docstring)."""
    prim_scale = max(np.max(np.abs(v)) if v.size else 0.0, np.max(np.abs(z_new)) if z_new.size else 0.0)
    hx, hu = H_apply(qp, x, u)
    gx, gu = GT_apply(qp, rho * y_new)
    qr = max(np.max(np.abs(qp.q)), np.max(np.abs(qp.r)) if qp.r.size else 0.0)
    dual_scale = max(np.max(np.abs(hx)), np.max(np.abs(hu)) if hu.size else 0.0,
                     np.max(np.abs(gx)), np.max(np.abs(gu)) if gu.size else 0.0, qr)
    if r_prim <= 0.0 or r_dual <= 0.0 or prim_scale <= 0.0 or dual_scale <= 0.0:
        return rho
    ratio = (r_prim / prim_scale) / (r_dual / dual_scale)
    return float(min(max(rho * np.sqrt(ratio), s.rho_min), s.rho_max))


def admm(qp, s: Settings | None = None, z0=None, y0=None, rho0=None, iters=None) -> Result:
    """ADMM per Sec. IV-A.  iters (if given) runs exactly that many
    iterations with no stop test (for iterate parity)."""
    s = s or Settings()
    qp0 = qp                       # original data: the KKT check always uses it
    refines = 0
    m = qp.m
    z = np.zeros(m) if z0 is None else np.array(z0, dtype=float)
    y = np.zeros(m) if y0 is None else np.array(y0, dtype=float)
    rho = s.rho0 if rho0 is None else float(rho0)
    eps = s.eps
    Qh, Rh, Sh = augmented(qp, rho)
    refactors = 1
    hist = [rho]
    max_iter = s.max_iter if iters is None else iters
    converged = False
    r_prim = r_dual = np.inf
    x = u = None
    kkt = None
    floor_it = -1                  # first stop-test iteration at the eps floor (stall rule)
    lam_ref = None                 # lambda one check interval before max_iter (certificate)
    t = 0
    for t in range(1, max_iter + 1):
        qh, rh = augmented_linear(qp, rho, y, z)
        x, u = lq_solve(qp, Qh, Rh, Sh, qh, rh, qp.x0)
        v = G_apply(qp, x, u)
        z_new = np.clip(v + y, qp.lo, qp.hi)
        y = y + v - z_new
        r_prim, r_dual = residuals(qp, v, z_new, z, rho)
        z = z_new
        if iters is not None:
            continue
        if t == max_iter - s.check_every:
            lam_ref = rho * y
        # eps counts as at the floor within a relative 1e-9: repeated
        # multiplication by 0.1 does not land on the floor exactly in binary
        at_floor = eps <= s.eps_floor * (1.0 + 1e-9)
        stalled = False
        if s.stall_iters > 0 and t % s.check_every == 0 and at_floor:
            if floor_it < 0:
                floor_it = t
            stalled = t - floor_it >= s.stall_iters
        if t % s.check_every == 0 and ((r_prim <= eps and r_dual <= eps) or stalled):
            floor_it = -1
            if s.eps_kkt is None:
                converged = True
                break
            kkt = kkt_residual(qp0, x, u, rho * y)
            if kkt <= s.eps_kkt:
                converged = True
                break
            if not at_floor:
                eps = max(eps * 0.1, s.eps_floor)
            elif refines < s.max_refine:
                qp = dataclasses.replace(qp, r=qp.r + u_residuals(qp0, x, u, rho * y))
                refines += 1
        if s.sigma and t % s.sigma == 0:
            rho_new = rho_rule(qp, x, u, v, z, y, rho, r_prim, r_dual, s)
            if rho_new > 5.0 * rho or rho_new < rho / 5.0:
                y = y * (rho / rho_new)
                rho = rho_new
                Qh, Rh, Sh = augmented(qp, rho)
                refactors += 1
                hist.append(rho)
    infeasible = False
    if iters is None and not converged and lam_ref is not None:
        # the iteration limit: classify by the certificate of oracle.infeas
        infeasible = certificate(qp0, rho * y - lam_ref, s.eps)["certified"]
    return Result(x=x, u=u, z=z, y=y, rho=rho, lam=rho * y, iters=t, r_prim=r_prim, r_dual=r_dual,
                  converged=converged, refactors=refactors, rho_hist=hist, kkt=kkt, infeasible=infeasible)


def exact_solution(qp, tol: float = 1e-11, max_iter: int = 200000):
    """Unique primal minimiser of eq. sqp_qp (Q, R > 0): ADMM driven to a tight
    tolerance, then a dense-KKT polish on the detected active set (oracle.activeset)."""
    from .activeset import polish
    r = admm(qp, Settings(eps=tol, sigma=25, check_every=5, max_iter=max_iter))
    return polish(qp, r.x, r.u, r.lam)
