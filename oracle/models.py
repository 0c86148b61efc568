"""The paper's analytic test models and the SQP / RTI outer loop around the
LTV-QP (Sec. III-B, Sec. IV-C, App. C, App. D).

Test infrastructure only (see oracle/__init__.py).

Models (state x, input u, time step dt):
  dubins   App. C: x = (p_x, p_y, theta), u = omega,
           f(x, u) = (p_x + v cos(theta) dt, p_y + v sin(theta) dt, theta + omega dt)
  quad2d   App. D: x = (p_x, p_y, phi, v_x, v_y, phidot), u = (u_1, u_2),
           xdot = (v_x, v_y, phidot, -(u_1 + u_2) sin(phi) / m,
                   (u_1 + u_2) cos(phi) / m - g, L (u_2 - u_1) / J),
           discretized by one explicit Euler step: f(x, u) = x + dt xdot.
Constraints: the input box u_lo <= u <= u_hi (two-sided rows) and, per
obstacle (c_x, c_y, r), r^2 - (p_x - c_x)^2 - (p_y - c_y)^2 <= 0 on every
stage and on x_N (eq. obstacle_constraints).
Cost: l(x, u) = 1/2 (x - x_ref)^T diag(Qd) (x - x_ref) + 1/2 (u - u_ref)^T diag(Rd) (u - u_ref),
      l_f(x) = 1/2 (x - x_ref)^T diag(QNd) (x - x_ref).

Readings (the paper is silent here):
  * the Hessian blocks of eq. sqp_qp use the cost Hessian alone
    (Gauss-Newton): the obstacle constraints are concave, and their curvature
    in the Lagrangian Hessian would make the QP nonconvex;
  * App. D gives continuous dynamics; one explicit Euler step discretizes them;
  * the step size alpha of Sec. III-B comes from a backtracking search on the
    l1 merit phi(X, U) = J + w (sum_k |f(x_k, u_k) - x_{k+1}|_1 + |x_0 - x0bar|_1
    + sum of constraint violations), alpha in {1, 1/2, ..., 1/128}, taking the
    first alpha with phi(alpha) < phi(0) (else the smallest);
  * RTI (Sec. IV-C): one linearization and one QP solve per control step, the
    full step (alpha = 1), the first input applied to the disturbed system
    x+ = f(x, u) + E w, and the nominal shifted by one stage (the last stage
    repeated) for the next step.
"""
from __future__ import annotations

import numpy as np

from paper_2604_07644_b300.workloads import QP
from paper_2604_07644_b300.workloads import ModelSpec as Model


def dynamics(m: Model, x, u):
    """x_{k+1} = f(x_k, u_k) (App. C; App. D with one Euler step)."""
    if m.kind == "dubins":
        return np.array([x[0] + m.v * np.cos(x[2]) * m.dt, x[1] + m.v * np.sin(x[2]) * m.dt, x[2] + u[0] * m.dt])
    T = u[0] + u[1]
    xdot = np.array([x[3], x[4], x[5], -T * np.sin(x[2]) / m.mass, T * np.cos(x[2]) / m.mass - m.grav,
                     m.arm * (u[1] - u[0]) / m.inertia])
    return x + m.dt * xdot


def jacobians(m: Model, x, u):
    """A = df/dx, B = df/du at (x, u), differentiated by hand from dynamics()."""
    if m.kind == "dubins":
        A = np.eye(3)
        A[0, 2] = -m.v * np.sin(x[2]) * m.dt
        A[1, 2] = m.v * np.cos(x[2]) * m.dt
        B = np.array([[0.0], [0.0], [m.dt]])
        return A, B
    T = u[0] + u[1]
    s, c = np.sin(x[2]), np.cos(x[2])
    Fx = np.zeros((6, 6))
    Fx[0, 3] = Fx[1, 4] = Fx[2, 5] = 1.0
    Fx[3, 2] = -T * c / m.mass
    Fx[4, 2] = -T * s / m.mass
    Fu = np.array([[0, 0], [0, 0], [0, 0], [-s / m.mass, -s / m.mass], [c / m.mass, c / m.mass],
                   [-m.arm / m.inertia, m.arm / m.inertia]])
    return np.eye(6) + m.dt * Fx, m.dt * Fu


def obstacle_g(m: Model, x):
    """g_o(x) = r^2 - (p_x - c_x)^2 - (p_y - c_y)^2 per obstacle (<= 0 is safe)."""
    o = m.obstacles
    return o[:, 2] ** 2 - (x[0] - o[:, 0]) ** 2 - (x[1] - o[:, 1]) ** 2


def obstacle_grad(m: Model, x):
    """Rows d g_o / dx: (-2 (p_x - c_x), -2 (p_y - c_y), 0, ...)."""
    o = m.obstacles
    G = np.zeros((m.n_obs, m.nx))
    G[:, 0] = -2.0 * (x[0] - o[:, 0])
    G[:, 1] = -2.0 * (x[1] - o[:, 1])
    return G


def linearize(m: Model, X, U, x0bar) -> QP:
    """The LTV-QP eq. sqp_qp in (dx, du) around the nominal (X, U):
    A_k, B_k the Jacobians; b_k = f(x_k, u_k) - x_{k+1} (the defect, so that
    x_{k+1} + dx_{k+1} = f(x_k, u_k) + A_k dx_k + B_k du_k); Gauss-Newton
    Q_k = diag(Qd), R_k = diag(Rd), S_k = 0, Q_N = diag(QNd); q_k, r_k, q_N the
    cost gradients at the nominal; stage rows [input box; obstacles] with
    C = (0; dg_o/dx), D = (I; 0), bounds (u_lo - u_k, u_hi - u_k) and
    (-inf, -g_o(x_k)); terminal obstacle rows likewise; dx_0 = x0bar - x_0."""
    N, nx, nu, no = m.N, m.nx, m.nu, m.n_obs
    nc = nu + no
    A = np.zeros((N, nx, nx))
    B = np.zeros((N, nx, nu))
    c = np.zeros((N, nx))
    C = np.zeros((N, nc, nx))
    D = np.zeros((N, nc, nu))
    lo = np.zeros(N * nc + no)
    hi = np.zeros(N * nc + no)
    q = np.zeros((N + 1, nx))
    r = np.zeros((N, nu))
    for k in range(N):
        A[k], B[k] = jacobians(m, X[k], U[k])
        c[k] = dynamics(m, X[k], U[k]) - X[k + 1]
        q[k] = m.Qd * (X[k] - m.xref)
        r[k] = m.Rd * (U[k] - m.uref)
        D[k, :nu] = np.eye(nu)
        C[k, nu:] = obstacle_grad(m, X[k])
        lo[k * nc:k * nc + nu] = m.u_lo - U[k]
        hi[k * nc:k * nc + nu] = m.u_hi - U[k]
        lo[k * nc + nu:(k + 1) * nc] = -np.inf
        hi[k * nc + nu:(k + 1) * nc] = -obstacle_g(m, X[k])
    q[N] = m.QNd * (X[N] - m.xref)
    CN = obstacle_grad(m, X[N])
    lo[N * nc:] = -np.inf
    hi[N * nc:] = -obstacle_g(m, X[N])
    Q = np.repeat(np.diag(m.Qd)[None], N + 1, axis=0)
    Q[N] = np.diag(m.QNd)
    R = np.repeat(np.diag(m.Rd)[None], N, axis=0)
    return QP(A=A, B=B, c=c, Q=Q, R=R, S=np.zeros((N, nu, nx)), q=q, r=r, C=C, D=D, CN=CN, lo=lo, hi=hi,
              x0=x0bar - X[0], name=f"{m.kind}-lin")


def cost(m: Model, X, U) -> float:
    J = 0.0
    for k in range(m.N):
        dxk, duk = X[k] - m.xref, U[k] - m.uref
        J += 0.5 * dxk @ (m.Qd * dxk) + 0.5 * duk @ (m.Rd * duk)
    dN = X[m.N] - m.xref
    return float(J + 0.5 * dN @ (m.QNd * dN))


def infeasibility(m: Model, X, U, x0bar) -> float:
    """sum_k |f(x_k, u_k) - x_{k+1}|_1 + |x_0 - x0bar|_1 + sum of constraint
    violations max(g, 0) and box violations."""
    s = float(np.sum(np.abs(X[0] - x0bar)))
    for k in range(m.N):
        s += float(np.sum(np.abs(dynamics(m, X[k], U[k]) - X[k + 1])))
        s += float(np.sum(np.maximum(U[k] - m.u_hi, 0.0) + np.maximum(m.u_lo - U[k], 0.0)))
        s += float(np.sum(np.maximum(obstacle_g(m, X[k]), 0.0)))
    s += float(np.sum(np.maximum(obstacle_g(m, X[m.N]), 0.0)))
    return s


def merit(m: Model, X, U, x0bar, w: float) -> float:
    return cost(m, X, U) + w * infeasibility(m, X, U, x0bar)


ALPHAS = [2.0 ** -i for i in range(8)]


def line_search(m: Model, X, U, dX, dU, x0bar, w: float):
    """First alpha in ALPHAS whose merit is below the merit at alpha = 0
    (else the smallest)."""
    phi0 = merit(m, X, U, x0bar, w)
    for a in ALPHAS:
        if merit(m, X + a * dX, U + a * dU, x0bar, w) < phi0:
            return a
    return ALPHAS[-1]


def sqp(m: Model, X, U, x0bar, iters: int, qp_solver, w: float = 100.0, line: bool = True):
    """`iters` SQP iterations (Sec. III-B) from the nominal (X, U): linearize,
    solve the LTV-QP (qp_solver(qp) -> (dx, du, lam)), step with alpha.
    Returns the list of (X, U, alpha, dx, du) after each iteration."""
    out = []
    X, U = X.copy(), U.copy()
    for _ in range(iters):
        qp = linearize(m, X, U, x0bar)
        dx, du, lam = qp_solver(qp)[:3]
        a = line_search(m, X, U, dx, du, x0bar, w) if line else 1.0
        X, U = X + a * dx, U + a * du
        out.append((X.copy(), U.copy(), a, dx, du))
    return out


def shift(X, U):
    """The nominal for the next control step: drop stage 0, repeat the last."""
    return np.concatenate([X[1:], X[-1:]]), np.concatenate([U[1:], U[-1:]])


def rti_rollout(m: Model, X, U, x0bar, W, qp_solver, tighten=None):
    """Closed loop of RTI steps (Sec. IV-C) under the disturbances W [steps, nx]
    (each step: x+ = f(x, u_0) + E w).  tighten(qp) -> qp, if given, applies
    the robust tightening to each step's QP.  Returns the visited states
    [steps + 1, nx], the applied inputs [steps, nu] and the final nominal."""
    xs = [x0bar.copy()]
    us = []
    X, U = X.copy(), U.copy()
    x = x0bar.copy()
    for w in W:
        qp = linearize(m, X, U, x)
        if tighten is not None:
            qp = tighten(qp)
        dx, du, lam = qp_solver(qp)[:3]
        X, U = X + dx, U + du
        u0 = U[0].copy()
        x = dynamics(m, x, u0) + m.E @ w
        xs.append(x.copy())
        us.append(u0)
        X, U = shift(X, U)
    return np.array(xs), np.array(us), (X, U)


def sls_problem(m: Model, qp: QP):
    """The SLS controller problem of a linearized step (eq. fastsls_qp):
    the QP's A_k, B_k, C_k, D_k, C_N, E_j = E, Qbar = Rbar = QbarN = I."""
    from paper_2604_07644_b300.workloads import SLSProblem
    N, nx, nu = m.N, m.nx, m.nu
    return SLSProblem(A=qp.A, B=qp.B, E=np.repeat(m.E[None], N, axis=0), Qbar=np.eye(nx), Rbar=np.eye(nu),
                      QbarN=np.eye(nx), C=qp.C, D=qp.D, CN=qp.CN, tau=None)


def rti_rollout_robust(m: Model, X, U, x0bar, W, qp_solver, eps: float = 1e-8):
    """RTI with the robust tightening of Sec. IV-C: each control step
    linearizes, updates the controller from the previous step's duals
    (zero at the first step), tightens, solves the tightened QP, takes the
    new duals (oracle.fastsls.step) and applies the first input to the
    disturbed plant.  Returns the visited states, the applied inputs and the
    margins of every step."""
    from . import fastsls
    xs = [x0bar.copy()]
    us, hs = [], []
    X, U = X.copy(), U.copy()
    x = x0bar.copy()
    tau = None
    for w in W:
        qp = linearize(m, X, U, x)
        s = fastsls.step(qp, sls_problem(m, qp), tau, eps, qp_solver)
        tau = s["tau"]
        X, U = X + s["x"], U + s["u"]
        u0 = U[0].copy()
        x = dynamics(m, x, u0) + m.E @ w
        xs.append(x.copy())
        us.append(u0)
        hs.append((s["h"], s["hf"]))
        X, U = shift(X, U)
    return np.array(xs), np.array(us), hs
