"""Seeded synthetic inputs for the LTV-QP and SLS workloads.

This module only draws problem data.  It holds none of the solver's arithmetic
(no Riccati step, no scan combine, no ADMM update), so both the CPU oracle and
the CUDA path may take their inputs from here.

Every draw goes through numpy's counter-based Philox bit generator keyed by the
seed, so a (workload, seed) pair always gives the same arrays on any machine.

Problem layout (row-major, time-major, float64), following the LTV-QP of
Sec. III-B (eq. sqp_qp):
    A  [N, nx, nx]   B [N, nx, nu]   c [N, nx]  (the paper's b_k)
    Q  [N+1, nx, nx] (Q[N] is the terminal Q_N)
    R  [N, nu, nu]   S [N, nu, nx]   q [N+1, nx]   r [N, nu]
    C  [N, nc, nx]   D [N, nc, nu]   CN [nf, nx]
    lo, hi [N*nc + nf]  two-sided bounds on G(dx, du); +-inf allowed
    x0 [nx]          the fixed initial state deviation
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

INF = float("inf")


def rng(*key: int) -> np.random.Generator:
    """Philox generator keyed by a tuple of non-negative ints (the tuple is
    hashed to the 128-bit Philox key by numpy's SeedSequence)."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(v) for v in key])))


@dataclass
class QP:
    """One horizon-structured, inequality-constrained LQ program."""
    A: np.ndarray
    B: np.ndarray
    c: np.ndarray
    Q: np.ndarray
    R: np.ndarray
    S: np.ndarray
    q: np.ndarray
    r: np.ndarray
    C: np.ndarray
    D: np.ndarray
    CN: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    x0: np.ndarray
    name: str = ""
    features: np.ndarray | None = None

    @property
    def nx(self) -> int:
        return self.A.shape[1]

    @property
    def nu(self) -> int:
        return self.B.shape[2]

    @property
    def N(self) -> int:
        return self.A.shape[0]

    @property
    def nc(self) -> int:
        return self.C.shape[1]

    @property
    def nf(self) -> int:
        return self.CN.shape[0]

    @property
    def m(self) -> int:
        """Number of constraint rows, N*nc + nf."""
        return self.N * self.nc + self.nf

    def dims(self) -> tuple[int, int, int, int, int]:
        return (self.nx, self.nu, self.N, self.nc, self.nf)


@dataclass
class SLSProblem:
    """Data of the SLS controller problem (eq. fastsls_qp) and its margins."""
    A: np.ndarray      # [N, nx, nx]
    B: np.ndarray      # [N, nx, nu]
    E: np.ndarray      # [N, nx, nx]   disturbance scaling E_j
    Qbar: np.ndarray   # [nx, nx]
    Rbar: np.ndarray   # [nu, nu]
    QbarN: np.ndarray  # [nx, nx]
    C: np.ndarray      # [N, nc, nx]
    D: np.ndarray      # [N, nc, nu]
    CN: np.ndarray     # [nf, nx]
    tau: np.ndarray | None = None  # [N+1, N, max(nc, nf)]; row k=N uses the first nf entries
    name: str = ""

    @property
    def nx(self) -> int:
        return self.A.shape[1]

    @property
    def nu(self) -> int:
        return self.B.shape[2]

    @property
    def N(self) -> int:
        return self.A.shape[0]

    @property
    def nc(self) -> int:
        return self.C.shape[1]

    @property
    def nf(self) -> int:
        return self.CN.shape[0]


# ----------------------------------------------------------------------------
# helpers (input construction only)
# ----------------------------------------------------------------------------

def _unit_rows(g: np.random.Generator, n_rows: int, dim: int) -> np.ndarray:
    M = g.standard_normal((n_rows, dim))
    return M / np.linalg.norm(M, axis=1, keepdims=True)


def _open_loop(A: np.ndarray, c: np.ndarray, x0: np.ndarray) -> np.ndarray:
    """Zero-input state sequence x_{k+1} = A_k x_k + c_k (problem data only)."""
    N, nx = A.shape[0], A.shape[1]
    X = np.zeros((N + 1, nx))
    X[0] = x0
    for k in range(N):
        X[k + 1] = A[k] @ X[k] + c[k]
    return X


def _raise_offsets(C: np.ndarray, hi: np.ndarray, X: np.ndarray, rows: np.ndarray, margin: float) -> None:
    """Raise one-sided offsets that the zero-input trajectory would come within
    `margin` of, so that u = 0 is strictly feasible (a feasibility guarantee by
    construction; rows lists the one-sided row indices of each stage)."""
    N = C.shape[0]
    nc = C.shape[1]
    for k in range(N):
        v = C[k] @ X[k]
        for i in rows:
            j = k * nc + i
            if v[i] + margin > hi[j]:
                hi[j] = v[i] + margin


def _empty(nx, nu, N):
    return dict(
        S=np.zeros((N, nu, nx)),
        c=np.zeros((N, nx)),
        r=np.zeros((N, nu)),
    )


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def plain_4d(seed: int = 0, N: int = 32) -> QP:
    """Plain FP64 QP: nx=4, nu=2, N=32, LTI A = I + 0.05 G, B ~ N(0, 0.1),
    Q = I, R = 0.1 I, |x| <= 5, |u| <= 1 (two-sided rows), terminal |x_N| <= 5,
    x0 ~ U[-2, 2]."""
    g = rng(1, seed)
    nx, nu = 4, 2
    # Rejection sampling on the problem data alone: redraw (G, x0) until the
    # zero-input trajectory stays inside |x| <= 4.5, which makes u = 0 a
    # strictly feasible point (with |u| <= 1 and B ~ 0.1, an unstable draw
    # would otherwise often be infeasible).
    for _ in range(1000):
        G = g.standard_normal((nx, nx))
        x0 = g.uniform(-2.0, 2.0, nx)
        A1 = np.eye(nx) + 0.05 * G
        X = _open_loop(np.repeat(A1[None], N, axis=0), np.zeros((N, nx)), x0)
        if np.max(np.abs(X)) <= 4.5:
            break
    Bm = 0.1 * g.standard_normal((nx, nu))
    A = np.repeat(A1[None], N, axis=0)
    B = np.repeat(Bm[None], N, axis=0)
    Q = np.repeat(np.eye(nx)[None], N + 1, axis=0)
    R = np.repeat(0.1 * np.eye(nu)[None], N, axis=0)
    C1 = np.vstack([np.eye(nx), np.zeros((nu, nx))])
    D1 = np.vstack([np.zeros((nx, nu)), np.eye(nu)])
    C = np.repeat(C1[None], N, axis=0)
    D = np.repeat(D1[None], N, axis=0)
    CN = np.eye(nx)
    nc = nx + nu
    hi = np.concatenate([np.tile(np.r_[5.0 * np.ones(nx), np.ones(nu)], N), 5.0 * np.ones(nx)])
    lo = -hi.copy()
    e = _empty(nx, nu, N)
    assert nc == C.shape[1]
    return QP(A=A, B=B, c=e["c"], Q=Q, R=R, S=e["S"], q=np.zeros((N + 1, nx)), r=e["r"],
              C=C, D=D, CN=CN, lo=lo, hi=hi, x0=x0, name=f"plain4d-N{N}-s{seed}")


def quadrotor_12d(seed: int = 0, N: int = 64) -> QP:
    """Quadrotor-shaped QP: nx=12, nu=4, N=64, A_k = I + 0.02 G_k,
    B_k ~ N(0, 0.05), Q = diag U[0.5, 2], R = diag U[0.01, 0.1], 24 unit
    half-spaces per stage on (x, u) with offsets U[1, 3], no terminal rows,
    x0 ~ U[-0.5, 0.5], a goal x_ref of norm 1.5 (q_k = -Q x_ref)."""
    g = rng(2, seed)
    nx, nu, nc = 12, 4, 24
    A = np.eye(nx)[None] + 0.02 * g.standard_normal((N, nx, nx))
    B = 0.05 * g.standard_normal((N, nx, nu))
    qd = g.uniform(0.5, 2.0, nx)
    rd = g.uniform(0.01, 0.1, nu)
    Q = np.repeat(np.diag(qd)[None], N + 1, axis=0)
    R = np.repeat(np.diag(rd)[None], N, axis=0)
    rows = _unit_rows(g, N * nc, nx + nu).reshape(N, nc, nx + nu)
    C = rows[:, :, :nx].copy()
    D = rows[:, :, nx:].copy()
    hi = np.concatenate([g.uniform(1.0, 3.0, N * nc), np.zeros(0)])
    lo = -INF * np.ones(N * nc)
    x0 = g.uniform(-0.5, 0.5, nx)
    xref = g.standard_normal(nx)
    xref *= 1.5 / np.linalg.norm(xref)
    q = -(Q @ xref)
    e = _empty(nx, nu, N)
    _raise_offsets(C, hi, _open_loop(A, e["c"], x0), np.arange(nc), 0.25)
    return QP(A=A, B=B, c=e["c"], Q=Q, R=R, S=e["S"], q=q, r=e["r"], C=C, D=D,
              CN=np.zeros((0, nx)), lo=lo, hi=hi, x0=x0, name=f"quad12d-N{N}-s{seed}")


def legged(seed: int = 0, nx: int = 61, nu: int = 12, N: int = 100, n_obs: int = 8,
           terminal_obstacles: bool = True, tag: int = 3) -> QP:
    """Legged-robot-shaped SQP inner QP (quadruped 61D/12u by default; the
    humanoid is nx=75, nu=21): A_k = I + 0.01 G_k, B_k ~ N(0, 0.02),
    Q = diag U[0.5, 2], R = diag U[0.01, 0.1]; per stage |u| <= 1 (nu two-sided
    rows) and n_obs unit half-spaces on the CoM plane (x_0, x_1) with offsets
    U[1, 3]; the same obstacle rows on x_N.  x0 ~ U[-0.5, 0.5]; a goal at radius
    2 in the CoM plane pulls the trajectory into the obstacles
    (q_k = -Q x_ref)."""
    g = rng(tag, seed, nx, N)
    A = np.eye(nx)[None] + 0.01 * g.standard_normal((N, nx, nx))
    B = 0.02 * g.standard_normal((N, nx, nu))
    qd = g.uniform(0.5, 2.0, nx)
    rd = g.uniform(0.01, 0.1, nu)
    Q = np.repeat(np.diag(qd)[None], N + 1, axis=0)
    R = np.repeat(np.diag(rd)[None], N, axis=0)
    nc = nu + n_obs
    C = np.zeros((N, nc, nx))
    D = np.zeros((N, nc, nu))
    D[:, :nu, :] = np.eye(nu)[None]
    dirs = _unit_rows(g, N * n_obs, 2).reshape(N, n_obs, 2)
    C[:, nu:, 0:2] = dirs
    f_obs = g.uniform(1.0, 3.0, (N, n_obs))
    hi_st = np.concatenate([np.ones((N, nu)), f_obs], axis=1)
    lo_st = np.concatenate([-np.ones((N, nu)), -INF * np.ones((N, n_obs))], axis=1)
    if terminal_obstacles:
        CN = np.zeros((n_obs, nx))
        CN[:, 0:2] = _unit_rows(g, n_obs, 2)
        fN = g.uniform(1.0, 3.0, n_obs)
    else:
        CN = np.zeros((0, nx))
        fN = np.zeros(0)
    hi = np.concatenate([hi_st.ravel(), fN])
    lo = np.concatenate([lo_st.ravel(), -INF * np.ones(CN.shape[0])])
    x0 = g.uniform(-0.5, 0.5, nx)
    phi = g.uniform(0.0, 2.0 * math.pi)
    xref = np.zeros(nx)
    xref[0], xref[1] = 2.0 * math.cos(phi), 2.0 * math.sin(phi)
    q = -(Q @ xref)
    e = _empty(nx, nu, N)
    X = _open_loop(A, e["c"], x0)
    _raise_offsets(C, hi, X, np.arange(nu, nc), 0.25)
    if CN.shape[0]:
        v = CN @ X[N]
        base = N * nc
        for i in range(CN.shape[0]):
            if v[i] + 0.25 > hi[base + i]:
                hi[base + i] = v[i] + 0.25
    return QP(A=A, B=B, c=e["c"], Q=Q, R=R, S=e["S"], q=q, r=e["r"], C=C, D=D,
              CN=CN, lo=lo, hi=hi, x0=x0, name=f"legged{nx}d-N{N}-s{seed}")


def quadruped_61d(seed: int = 0, N: int = 100) -> QP:
    """Quadruped-shaped inner QP: nx=61, nu=12, N=100, nc=20 (12 box + 8
    obstacles), nf=8."""
    return legged(seed, 61, 12, N)


def humanoid_75d(seed: int = 0, N: int = 40) -> QP:
    """Humanoid-shaped QP: nx=75, nu=21, N=40, nc=29, nf=8."""
    return legged(seed, 75, 21, N, tag=4)


def infeasible_x0(seed: int = 0) -> QP:
    """The plain 4D QP with x0[0] = 9: x_0 = x0 is fixed and violates the
    stage-0 state bound |x| <= 5, so no feasible point exists."""
    qp = plain_4d(seed)
    x0 = qp.x0.copy()
    x0[0] = 9.0
    return dataclasses.replace(qp, x0=x0, name=f"infeasible-x0-s{seed}")


def infeasible_terminal(seed: int = 1, N: int = 12) -> QP:
    """The plain 4D QP with |u| <= 1e-3 and the terminal row x_N[0] pinned to
    4.9, which the nearly open-loop trajectory from x0 (kept inside |x| <= 4.5
    by the plain 4D draw) cannot reach: no feasible point exists."""
    qp = plain_4d(seed, N=N)
    nx, nc = qp.nx, qp.nc
    lo, hi = qp.lo.copy(), qp.hi.copy()
    for k in range(N):
        lo[k * nc + nx:(k + 1) * nc] = -1e-3   # rows [x; u]: the u rows
        hi[k * nc + nx:(k + 1) * nc] = 1e-3
    lo[N * nc], hi[N * nc] = 4.9, 4.9
    return dataclasses.replace(qp, lo=lo, hi=hi, name=f"infeasible-terminal-s{seed}")


def long_horizon(seed: int = 0, links: int = 15, N: int = 3000, dt: float = 0.01) -> QP:
    """Long-horizon workload shaped like a torque-limited n-link pendulum
    linearized along a trajectory (Sec. V-A's horizon study: more than 1.35e5
    decision variables at N = 3000, i.e. nx + nu = 45 per stage): state
    (angles, rates), nx = 2 links, nu = links,
        A_k = [[I, dt I], [-dt K_k, I - dt Dmp]],  B_k = [[0], [dt M^-1]],
    with a chain stiffness K_k = diag(s) + 0.5 L (L the path Laplacian,
    s ~ U[0.5, 1.5]) plus a symmetric per-stage perturbation 0.05 sym(G_k),
    damping Dmp = 0.1 I, M^-1 = I + 0.05 sym(G); Q = diag(U[1, 5] on angles,
    U[0.05, 0.2] on rates), Q_N = Q, R = diag U[0.01, 0.1]; torque limits
    |u| <= 1 (nc = nu two-sided rows), no terminal rows; angle targets of
    +-1 rad (q_k = -Q x_ref) that the torque limits make active;
    x0 = (U[-0.5, 0.5] angles, zero rates)."""
    g = rng(14, seed, links, N)
    n = links
    nx, nu = 2 * n, n
    lap = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    lap[0, 0] = lap[-1, -1] = 1.0
    Kc = np.diag(g.uniform(0.5, 1.5, n)) + 0.5 * lap
    Gm = g.standard_normal((n, n))
    Minv = np.eye(n) + 0.05 * (Gm + Gm.T) / 2.0
    A = np.zeros((N, nx, nx))
    B = np.zeros((N, nx, nu))
    Gk = g.standard_normal((N, n, n))
    for k in range(N):
        Kk = Kc + 0.05 * (Gk[k] + Gk[k].T) / 2.0
        A[k, :n, :n] = np.eye(n)
        A[k, :n, n:] = dt * np.eye(n)
        A[k, n:, :n] = -dt * Kk
        A[k, n:, n:] = (1.0 - 0.1 * dt) * np.eye(n)
        B[k, n:, :] = dt * Minv
    qd = np.concatenate([g.uniform(1.0, 5.0, n), g.uniform(0.05, 0.2, n)])
    rd = g.uniform(0.01, 0.1, nu)
    Q = np.repeat(np.diag(qd)[None], N + 1, axis=0)
    R = np.repeat(np.diag(rd)[None], N, axis=0)
    C = np.zeros((N, nu, nx))
    D = np.repeat(np.eye(nu)[None], N, axis=0)
    hi = np.ones(N * nu)
    lo = -hi.copy()
    xref = np.concatenate([np.where(np.arange(n) % 2 == 0, 1.0, -1.0), np.zeros(n)])
    q = np.repeat(-(np.diag(qd) @ xref)[None], N + 1, axis=0)
    x0 = np.concatenate([g.uniform(-0.5, 0.5, n), np.zeros(n)])
    e = _empty(nx, nu, N)
    return QP(A=A, B=B, c=e["c"], Q=Q, R=R, S=e["S"], q=q, r=e["r"], C=C, D=D, CN=np.zeros((0, nx)), lo=lo, hi=hi,
              x0=x0, name=f"pendulum{n}-N{N}-s{seed}")


def tiny(seed: int = 0, nx: int = 2, nu: int = 1, N: int = 3, box_u: float = 0.3,
         n_half: int = 1, S_nonzero: bool = True, b_nonzero: bool = True) -> QP:
    """Tiny random QP for brute-force pins: dense random A, B, SPD Q, R, random
    S (small enough that the stage Hessian stays SPD), affine term b, two-sided
    |u| <= box_u rows and n_half random half-spaces per stage, one terminal
    half-space."""
    g = rng(9, seed, nx, nu, N)
    A = g.standard_normal((N, nx, nx)) * 0.6 + np.eye(nx)[None] * 0.5
    B = g.standard_normal((N, nx, nu))
    Q = np.zeros((N + 1, nx, nx))
    R = np.zeros((N, nu, nu))
    S = np.zeros((N, nu, nx))
    for k in range(N + 1):
        M = g.standard_normal((nx, nx))
        Q[k] = M @ M.T / nx + 0.5 * np.eye(nx)
    for k in range(N):
        M = g.standard_normal((nu, nu))
        R[k] = M @ M.T / nu + 0.5 * np.eye(nu)
        if S_nonzero:
            S[k] = 0.2 * g.standard_normal((nu, nx))
    c = 0.3 * g.standard_normal((N, nx)) if b_nonzero else np.zeros((N, nx))
    q = g.standard_normal((N + 1, nx))
    r = g.standard_normal((N, nu))
    nc = nu + n_half
    C = np.zeros((N, nc, nx))
    D = np.zeros((N, nc, nu))
    D[:, :nu, :] = np.eye(nu)[None]
    rows = _unit_rows(g, N * n_half, nx + nu).reshape(N, n_half, nx + nu)
    C[:, nu:, :] = rows[:, :, :nx]
    D[:, nu:, :] = rows[:, :, nx:]
    f = g.uniform(0.2, 1.0, (N, n_half))
    hi = np.concatenate([np.concatenate([box_u * np.ones((N, nu)), f], axis=1).ravel(),
                         g.uniform(0.5, 1.5, 1)])
    lo = np.concatenate([np.concatenate([-box_u * np.ones((N, nu)), -INF * np.ones((N, n_half))], axis=1).ravel(),
                         -INF * np.ones(1)])
    CN = _unit_rows(g, 1, nx)
    x0 = g.uniform(-0.5, 0.5, nx)
    X = _open_loop(A, c, x0)
    _raise_offsets(C, hi, X, np.arange(nu, nc), 0.2)
    v = CN @ X[N]
    if v[0] + 0.2 > hi[N * nc]:
        hi[N * nc] = v[0] + 0.2
    return QP(A=A, B=B, c=c, Q=Q, R=R, S=S, q=q, r=r, C=C, D=D, CN=CN, lo=lo, hi=hi,
              x0=x0, name=f"tiny-{nx}-{nu}-{N}-s{seed}")


def random_general(seed: int, nx: int, nu: int, N: int, nc: int, nf: int,
                   active_scale: float = 1.0) -> QP:
    """General random QP with every term present (S, b, q, r nonzero, two-sided
    and one-sided rows); used for kernel parity across ragged sizes."""
    g = rng(11, seed, nx, nu, N)
    A = np.eye(nx)[None] + 0.1 * g.standard_normal((N, nx, nx)) / math.sqrt(nx)
    B = 0.3 * g.standard_normal((N, nx, nu))
    Q = np.zeros((N + 1, nx, nx))
    R = np.zeros((N, nu, nu))
    S = np.zeros((N, nu, nx))
    for k in range(N + 1):
        M = g.standard_normal((nx, nx)) / math.sqrt(nx)
        Q[k] = M @ M.T + 0.5 * np.eye(nx)
    for k in range(N):
        M = g.standard_normal((nu, nu)) / math.sqrt(nu)
        R[k] = M @ M.T + 0.5 * np.eye(nu)
        S[k] = 0.1 * g.standard_normal((nu, nx))
    c = 0.05 * g.standard_normal((N, nx))
    q = 0.5 * g.standard_normal((N + 1, nx))
    r = 0.5 * g.standard_normal((N, nu))
    rows = _unit_rows(g, N * nc, nx + nu).reshape(N, nc, nx + nu) if nc else np.zeros((N, 0, nx + nu))
    C = rows[:, :, :nx].copy()
    D = rows[:, :, nx:].copy()
    CN = _unit_rows(g, nf, nx) if nf else np.zeros((0, nx))
    hi_st = g.uniform(0.3, 1.0, (N, nc)) * active_scale
    lo_st = -g.uniform(0.3, 1.0, (N, nc)) * active_scale
    # every third row one-sided (lo = -inf)
    lo_st[:, ::3] = -INF
    hi = np.concatenate([hi_st.ravel(), g.uniform(0.5, 1.5, nf)])
    lo = np.concatenate([lo_st.ravel(), -INF * np.ones(nf)])
    x0 = g.uniform(-0.3, 0.3, nx)
    X = _open_loop(A, c, x0)
    for k in range(N):
        v = C[k] @ X[k]
        for i in range(nc):
            j = k * nc + i
            if v[i] + 0.2 > hi[j]:
                hi[j] = v[i] + 0.2
            if v[i] - 0.2 < lo[j]:
                lo[j] = v[i] - 0.2
    if nf:
        v = CN @ X[N]
        for i in range(nf):
            j = N * nc + i
            if v[i] + 0.2 > hi[j]:
                hi[j] = v[i] + 0.2
    return QP(A=A, B=B, c=c, Q=Q, R=R, S=S, q=q, r=r, C=C, D=D, CN=CN, lo=lo, hi=hi,
              x0=x0, name=f"general-{nx}-{nu}-{N}-{nc}-{nf}-s{seed}")


def serving_mix(seed: int = 0, count: int = 256) -> list[QP]:
    """Batched serving mix: nx family uniform over (12,4)/(61,12)/(75,21),
    N ~ U{16..128}; 12D drawn as the quadrotor recipe, 61D/75D as the legged
    recipe."""
    g = rng(5, seed)
    out = []
    for i in range(count):
        fam = int(g.integers(0, 3))
        N = int(g.integers(16, 129))
        s = int(g.integers(0, 2**31 - 1))
        if fam == 0:
            out.append(quadrotor_12d(s, N))
        elif fam == 1:
            out.append(legged(s, 61, 12, N))
        else:
            out.append(legged(s, 75, 21, N, tag=4))
    return out


# ----------------------------------------------------------------------------
# learned warm-start family: one base linearization, per-instance x0 and a
# low-dimensional perturbation theta of the linearization and the goal
# ----------------------------------------------------------------------------

N_THETA = 8


@dataclass
class Family:
    base: QP
    M: np.ndarray = field(repr=False)        # [N_THETA, nx, nx] perturbation directions of A
    goal_dirs: np.ndarray = field(repr=False)  # [N_THETA, 2]

    def instance(self, i: int, N: int | None = None) -> QP:
        """Instance i: x0 ~ U[-0.5, 0.5]^nx, theta ~ U[-1, 1]^8,
        A_k(theta) = A_k + 0.002 sum_l theta_l M_l, goal angle set by theta.
        N (<= the base horizon): the first N stages of the base problem with
        its terminal cost and rows (the serving mix's ragged horizons)."""
        b = self.base if N is None or N == self.base.N else _truncate(self.base, N)
        g = rng(77, i, b.nx)
        x0 = g.uniform(-0.5, 0.5, b.nx)
        th = g.uniform(-1.0, 1.0, N_THETA)
        dA = 0.002 * np.tensordot(th, self.M, axes=(0, 0))
        A = b.A + dA[None]
        gd = th @ self.goal_dirs
        xref = np.zeros(b.nx)
        nrm = np.linalg.norm(gd)
        gd = gd / nrm if nrm > 1e-9 else np.array([1.0, 0.0])
        xref[0], xref[1] = 2.0 * gd[0], 2.0 * gd[1]
        q = -(b.Q @ xref)
        hi = b.hi.copy()
        X = _open_loop(A, b.c, x0)
        nc = b.nc
        one_sided = [i for i in range(nc) if not np.isfinite(b.lo[i])]
        _raise_offsets(b.C, hi, X, np.array(one_sided, dtype=int), 0.25)
        if b.nf:
            v = b.CN @ X[b.N]
            for j in range(b.nf):
                jj = b.N * nc + j
                if v[j] + 0.25 > hi[jj]:
                    hi[jj] = v[j] + 0.25
        return QP(A=A, B=b.B, c=b.c, Q=b.Q, R=b.R, S=b.S, q=q, r=b.r, C=b.C, D=b.D,
                  CN=b.CN, lo=b.lo, hi=hi, x0=x0, name=f"{b.name}-inst{i}",
                  features=np.concatenate([x0, th]))


def _truncate(qp: QP, N: int) -> QP:
    """The first N stages of qp with its terminal cost and terminal rows."""
    if not 1 <= N <= qp.N:
        raise ValueError("horizon out of range")
    nc = qp.nc
    return QP(A=qp.A[:N], B=qp.B[:N], c=qp.c[:N], Q=np.concatenate([qp.Q[:N], qp.Q[-1:]]), R=qp.R[:N],
              S=qp.S[:N], q=np.concatenate([qp.q[:N], qp.q[-1:]]), r=qp.r[:N], C=qp.C[:N], D=qp.D[:N], CN=qp.CN,
              lo=np.concatenate([qp.lo[:N * nc], qp.lo[qp.N * nc:]]),
              hi=np.concatenate([qp.hi[:N * nc], qp.hi[qp.N * nc:]]), x0=qp.x0, name=f"{qp.name}-N{N}")


def family_from(base: QP, seed: int) -> Family:
    """A warm-start family around any base problem (the perturbation
    directions M_l and goal directions drawn from the seed)."""
    nx = base.nx
    g = rng(79, seed, nx)
    M = g.standard_normal((N_THETA, nx, nx)) / math.sqrt(nx)
    goal_dirs = g.standard_normal((N_THETA, 2))
    return Family(base=base, M=M, goal_dirs=goal_dirs)


# shape families of the serving mix (nx, nu): the quadrotor-shaped 12D/4 and
# the legged 61D/12 and 75D/21 recipes, each built at the longest horizon
# (128) and truncated per instance
MIX_FAMILIES = ((12, 4), (61, 12), (75, 21))
MIX_N_MAX = 128


def mix_family(kind: int, seed: int = 0) -> Family:
    """Family `kind` (0: 12D quadrotor-shaped, 1: 61D, 2: 75D legged) of
    the learned serving mix, at horizon MIX_N_MAX."""
    if kind == 0:
        return family_from(quadrotor_12d(seed + 1000, MIX_N_MAX), seed)
    nx, nu = MIX_FAMILIES[kind]
    return family_from(legged(seed + 1000, nx, nu, MIX_N_MAX, tag=6 + kind), seed + kind)


def serving_mix_learned(seed: int = 0, count: int = 256, first: int = 100000):
    """256 QPs of the three mix families (uniform) with N ~ U{16..128}, as
    (QP, family kind) pairs; instance indices from `first` (held out from
    training, which uses indices below 100000)."""
    g = rng(23, seed, count)
    fams = [mix_family(k) for k in range(3)]
    out = []
    for i in range(count):
        kind = int(g.integers(0, 3))
        N = int(g.integers(16, MIX_N_MAX + 1))
        out.append((fams[kind].instance(first + i, N), kind))
    return out


def family(seed: int = 0, nx: int = 61, nu: int = 12, N: int = 100) -> Family:
    base = legged(seed, nx, nu, N, tag=6)
    g = rng(78, seed, nx)
    M = g.standard_normal((N_THETA, nx, nx)) / math.sqrt(nx)
    goal_dirs = g.standard_normal((N_THETA, 2))
    return Family(base=base, M=M, goal_dirs=goal_dirs)


# ----------------------------------------------------------------------------
# SLS workloads
# ----------------------------------------------------------------------------

def sls_problem(seed: int = 0, nx: int = 75, nu: int = 21, N: int = 40, n_obs: int = 8,
                tau_mode: str = "zero") -> SLSProblem:
    """Humanoid-shaped SLS reachability problem generated as the legged QP:
    E = diag U[0.001, 0.01] (time-invariant), Qbar = I, Rbar = I, QbarN = I;
    tau either zero (None) or U[0, 1] per (k, j, row)."""
    qp = legged(seed, nx, nu, N, n_obs, tag=4)
    g = rng(8, seed, nx, N)
    w = g.uniform(0.001, 0.01, nx)
    E = np.repeat(np.diag(w)[None], N, axis=0)
    tau = None
    if tau_mode == "uniform":
        tau = g.uniform(0.0, 1.0, (N + 1, N, max(qp.nc, qp.nf)))
    return SLSProblem(A=qp.A, B=qp.B, E=E, Qbar=np.eye(nx), Rbar=np.eye(nu), QbarN=np.eye(nx),
                      C=qp.C, D=qp.D, CN=qp.CN, tau=tau, name=f"sls{nx}d-N{N}-{tau_mode}-s{seed}")


def fastsls_problem(seed: int = 0, nx: int = 12, nu: int = 4, N: int = 17, n_obs: int = 8,
                    w_range: tuple = (0.002, 0.01), tag: int = 12) -> tuple[QP, SLSProblem]:
    """Nominal LTV-QP and SLS controller data of the FastSLS alternation
    (Sec. III-D) sharing A_k, B_k, C_k, D_k, C_N: the legged recipe (|u| <= 1
    box rows and obstacle half-spaces that the goal pulls the trajectory
    into), E = diag(w) with w ~ U[w_range] per state (time-invariant),
    Qbar = I, Rbar = I, QbarN = I.  tag 4 with (75, 21, 40) and w in
    [0.001, 0.01] is the humanoid-shaped problem of sls_problem."""
    qp = legged(seed, nx, nu, N, n_obs, tag=tag)
    g = rng(13, seed, nx, N)
    w = g.uniform(w_range[0], w_range[1], nx)
    E = np.repeat(np.diag(w)[None], N, axis=0)
    sp = SLSProblem(A=qp.A, B=qp.B, E=E, Qbar=np.eye(nx), Rbar=np.eye(nu), QbarN=np.eye(nx), C=qp.C, D=qp.D,
                    CN=qp.CN, tau=None, name=f"fastsls{nx}d-N{N}-s{seed}")
    return qp, sp


def sls_small(seed: int = 0, nx: int = 3, nu: int = 2, N: int = 5, nc: int = 3, nf: int = 2,
              tau_mode: str = "uniform") -> SLSProblem:
    """Small random SLS problem for pins and parity (every term present)."""
    g = rng(10, seed, nx, nu, N)
    A = np.eye(nx)[None] + 0.3 * g.standard_normal((N, nx, nx))
    B = g.standard_normal((N, nx, nu))
    E = 0.1 * g.standard_normal((N, nx, nx))
    M = g.standard_normal((nx, nx))
    Qbar = M @ M.T / nx + 0.5 * np.eye(nx)
    M = g.standard_normal((nu, nu))
    Rbar = M @ M.T / nu + 0.5 * np.eye(nu)
    M = g.standard_normal((nx, nx))
    QbarN = M @ M.T / nx + 0.5 * np.eye(nx)
    C = g.standard_normal((N, nc, nx))
    D = g.standard_normal((N, nc, nu))
    CN = g.standard_normal((nf, nx))
    tau = g.uniform(0.0, 1.0, (N + 1, N, max(nc, nf))) if tau_mode == "uniform" else None
    return SLSProblem(A=A, B=B, E=E, Qbar=Qbar, Rbar=Rbar, QbarN=QbarN, C=C, D=D, CN=CN,
                      tau=tau, name=f"sls-small-{nx}-{nu}-{N}-s{seed}")


# ----------------------------------------------------------------------------
# analytic models of App. C (Dubins car) and App. D (planar quadrotor) for
# the SQP / RTI outer loop: parameters, references, weights, obstacles and
# disturbance draws (data only; the dynamics live in the oracle and the
# library)
# ----------------------------------------------------------------------------

MODEL_DUBINS, MODEL_QUAD2D = 0, 1
MODEL_MAX_OBS = 16


@dataclass
class ModelSpec:
    """One model instance: kind ("dubins" / "quad2d"), horizon N, time step,
    obstacles [n_obs, 3] (c_x, c_y, r), input box, tracking reference and
    diagonal weights (stage Qd, Rd; terminal QNd), disturbance scaling E and
    the physical parameters (Dubins speed v; quadrotor m, g, L, J of App. D)."""
    kind: str
    N: int
    dt: float
    obstacles: np.ndarray
    u_lo: np.ndarray
    u_hi: np.ndarray
    xref: np.ndarray
    uref: np.ndarray
    Qd: np.ndarray
    Rd: np.ndarray
    QNd: np.ndarray
    E: np.ndarray
    x0: np.ndarray
    v: float = 1.0
    mass: float = 2.0576
    grav: float = 9.81
    arm: float = 0.25
    inertia: float = 0.01

    @property
    def nx(self) -> int:
        return 3 if self.kind == "dubins" else 6

    @property
    def nu(self) -> int:
        return 1 if self.kind == "dubins" else 2

    @property
    def n_obs(self) -> int:
        return self.obstacles.shape[0]

    def dims(self) -> tuple[int, int, int, int, int]:
        return (self.nx, self.nu, self.N, self.nu + self.n_obs, self.n_obs)

    def initial_guess(self) -> tuple[np.ndarray, np.ndarray]:
        """Nominal to start SQP from: the state held at x0, inputs at u_ref;
        for the Dubins car the states after x0 follow the chord from x0 to
        the reference position at speed v, heading along it."""
        X = np.repeat(self.x0[None], self.N + 1, axis=0)
        if self.kind == "dubins":
            d = self.xref[:2] - self.x0[:2]
            th = float(np.arctan2(d[1], d[0]))
            t = np.arange(1, self.N + 1) * self.dt * self.v
            X[1:, 0] = self.x0[0] + t * np.cos(th)
            X[1:, 1] = self.x0[1] + t * np.sin(th)
            X[1:, 2] = th
        U = np.repeat(self.uref[None], self.N, axis=0)
        return X, U


def dubins(seed: int = 0, N: int = 30, n_obs: int = 2) -> ModelSpec:
    """Dubins car of App. C: v = 1 m/s, dt = 0.1 s, |omega| <= 2, from the
    origin heading +x towards a goal at (2.6, 1.2) (the chord to it is
    shorter than the N dt v = 3 m path, so the car must turn) past obstacles
    of radius U[0.3, 0.45] whose edges sit 0.05 to 0.15 m from the chord, on
    alternating sides; E = 2.5e-2 I_3."""
    g = rng(20, seed, N)
    goal = np.array([2.6, 1.2])
    d = goal / np.linalg.norm(goal)
    nrm = np.array([-d[1], d[0]])
    obs = np.zeros((n_obs, 3))
    for i in range(n_obs):
        r = g.uniform(0.3, 0.45)
        side = 1.0 if i % 2 == 0 else -1.0
        s_ = (0.35 + 0.4 * i / max(1, n_obs - 1) + g.uniform(-0.05, 0.05)) * np.linalg.norm(goal)
        cxy = s_ * d + side * (r + g.uniform(0.05, 0.15)) * nrm
        obs[i] = [cxy[0], cxy[1], r]
    return ModelSpec(kind="dubins", N=N, dt=0.1, obstacles=obs, u_lo=np.array([-2.0]), u_hi=np.array([2.0]),
                     xref=np.array([goal[0], goal[1], 0.0]), uref=np.zeros(1), Qd=np.array([1.0, 1.0, 0.1]),
                     Rd=np.array([0.1]), QNd=np.array([10.0, 10.0, 1.0]), E=2.5e-2 * np.eye(3),
                     x0=np.zeros(3), v=1.0)


def quad2d(seed: int = 0, N: int = 40, n_obs: int = 1) -> ModelSpec:
    """Planar quadrotor of App. D (m = 2.0576, g = 9.81, L = 0.25, J = 0.01),
    dt = 0.05 s, thrusts 0 <= u_i <= 20, from hover at the origin to a goal
    at (2, 0) past obstacles of radius U[0.3, 0.4] whose edges sit 0.05 to
    0.15 m from the straight path; E = 5e-2 diag(0, 0, 0, 1, 1, 0)."""
    g = rng(21, seed, N)
    mass, grav = 2.0576, 9.81
    uh = mass * grav / 2.0
    obs = np.zeros((n_obs, 3))
    for i in range(n_obs):
        r = g.uniform(0.3, 0.4)
        side = 1.0 if i % 2 == 0 else -1.0
        obs[i] = [1.0 + g.uniform(-0.2, 0.2) + 0.6 * i, side * (r + g.uniform(0.05, 0.15)), r]
    Qd = np.array([5.0, 5.0, 1.0, 1.0, 1.0, 0.1])
    return ModelSpec(kind="quad2d", N=N, dt=0.05, obstacles=obs, u_lo=np.zeros(2), u_hi=np.array([20.0, 20.0]),
                     xref=np.array([2.0, 0.0, 0.0, 0.0, 0.0, 0.0]), uref=np.array([uh, uh]), Qd=Qd,
                     Rd=np.array([0.1, 0.1]), QNd=10.0 * Qd, E=5e-2 * np.diag([0.0, 0, 0, 1, 1, 0]),
                     x0=np.zeros(6), mass=mass, grav=grav)


def disturbances(seed: int, steps: int, batch: int, nx: int) -> np.ndarray:
    """Disturbance draws w [steps, batch, nx] in the unit ball (|w|_2 <= 1,
    direction uniform, radius U[0, 1]^(1/nx))."""
    g = rng(22, seed, steps, batch, nx)
    w = g.standard_normal((steps, batch, nx))
    w /= np.linalg.norm(w, axis=2, keepdims=True)
    return w * g.uniform(0.0, 1.0, (steps, batch, 1)) ** (1.0 / nx)


# ----------------------------------------------------------------------------
# MLP initial weights (input to both the GPU trainer and the oracle)
# ----------------------------------------------------------------------------

def mlp_init(n_in: int, hidden: int, n_out: int, seed: int = 0):
    """He-uniform initial weights [W1, b1, W2, b2, W3, b3] (float64); the last
    layer is scaled by 0.1 so that an untrained network predicts near zero."""
    g = rng(1234, seed, n_in, n_out)

    def lin(o, i):
        lim = np.sqrt(6.0 / i)
        return g.uniform(-lim, lim, (o, i)), np.zeros(o)

    W1, b1 = lin(hidden, n_in)
    W2, b2 = lin(hidden, hidden)
    W3, b3 = lin(n_out, hidden)
    W3 *= 0.1
    return [W1, b1, W2, b2, W3, b3]
