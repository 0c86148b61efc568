"""Pins of the oracle's LQ pieces (not gpu)."""
import math

import numpy as np
import pytest

from oracle import lq
from paper_2604_07644_b300 import workloads as W


def _aug_random(qp, rho, seed):
    g = np.random.default_rng(seed)
    Qh, Rh, Sh = lq.augmented(qp, rho)
    y = g.standard_normal(qp.m)
    z = g.standard_normal(qp.m)
    qh, rh = lq.augmented_linear(qp, rho, y, z)
    return Qh, Rh, Sh, qh, rh


@pytest.mark.parametrize("dims", [(2, 1, 3, 2, 1), (3, 2, 6, 4, 2), (5, 3, 10, 6, 3)])
@pytest.mark.parametrize("seed", [0, 1])
def test_riccati_equals_dense_kkt(dims, seed):
    """The sequential Riccati solve of eq. primal_update equals the dense KKT
    solve of the same equality-constrained QP (S != 0, b != 0, q, r != 0)."""
    qp = W.random_general(seed, *dims)
    Qh, Rh, Sh, qh, rh = _aug_random(qp, 0.37, seed)
    x, u = lq.lq_solve(qp, Qh, Rh, Sh, qh, rh, qp.x0)
    xd, ud, _ = lq.dense_kkt_lq(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh, qp.x0)
    assert np.allclose(x, xd, atol=1e-11, rtol=0)
    assert np.allclose(u, ud, atol=1e-11, rtol=0)


def test_augmented_is_quadratic_penalty():
    """Q^, R^, S^ (eq. augmented_matrices, S^ = S + rho D^T C) are the Hessian
    of J + rho/2 ||G xi||^2: check against finite differences of the penalised
    objective on a random point."""
    qp = W.random_general(3, 3, 2, 4, 3, 2)
    rho = 0.8
    Qh, Rh, Sh = lq.augmented(qp, rho)
    g = np.random.default_rng(0)
    x = g.standard_normal((qp.N + 1, qp.nx))
    u = g.standard_normal((qp.N, qp.nu))

    def pen(x, u):
        v = lq.G_apply(qp, x, u)
        J = lq.objective(qp, x, u) - sum(qp.q[k] @ x[k] for k in range(qp.N + 1)) - \
            sum(qp.r[k] @ u[k] for k in range(qp.N))
        return J + 0.5 * rho * v @ v

    def quad(x, u):
        J = 0.0
        for k in range(qp.N):
            J += 0.5 * x[k] @ Qh[k] @ x[k] + u[k] @ Sh[k] @ x[k] + 0.5 * u[k] @ Rh[k] @ u[k]
        return J + 0.5 * x[qp.N] @ Qh[qp.N] @ x[qp.N]

    assert abs(pen(x, u) - quad(x, u)) < 1e-10 * max(1.0, abs(quad(x, u)))


@pytest.mark.parametrize("a,b,q,r", [(1.2, 0.5, 1.0, 0.3), (0.7, 1.1, 2.0, 0.05), (1.0, 1.0, 1.0, 1.0)])
def test_scalar_dare_closed_form(a, b, q, r):
    """Scalar LTI problem at long horizon: P_0 converges to the positive root of
    b^2 P^2 + (r - a^2 r - q b^2) P - q r = 0 (discrete algebraic Riccati)."""
    N = 400
    A = np.full((N, 1, 1), a)
    B = np.full((N, 1, 1), b)
    Q = np.full((N + 1, 1, 1), q)
    R = np.full((N, 1, 1), r)
    S = np.zeros((N, 1, 1))
    P, p, K, kff, G = lq.riccati(A, B, np.zeros((N, 1)), Q, R, S, np.zeros((N + 1, 1)), np.zeros((N, 1)))
    A2, B2, C2 = b * b, r - a * a * r - q * b * b, -q * r
    root = (-B2 + math.sqrt(B2 * B2 - 4 * A2 * C2)) / (2 * A2)
    assert abs(P[0, 0, 0] - root) < 1e-10 * max(1.0, root)
    # LQR gain closed form K = -a b P / (r + b^2 P)
    assert abs(K[0, 0, 0] + a * b * root / (r + b * b * root)) < 1e-10


def test_unconstrained_is_lqr_rollout():
    """With nc = nf = 0 the QP is plain LQR: Riccati rollout equals the dense
    KKT minimiser and the objective is below that of random feasible
    trajectories."""
    qp = W.random_general(5, 4, 2, 8, 0, 0)
    x, u = lq.lq_solve(qp, qp.Q, qp.R, qp.S, qp.q, qp.r, qp.x0)
    J = lq.objective(qp, x, u)
    g = np.random.default_rng(1)
    for _ in range(20):
        du = u + 0.1 * g.standard_normal(u.shape)
        xx = np.zeros_like(x)
        xx[0] = qp.x0
        for k in range(qp.N):
            xx[k + 1] = qp.A[k] @ xx[k] + qp.B[k] @ du[k] + qp.c[k]
        assert lq.objective(qp, xx, du) > J


def test_planted_mistake_in_riccati_is_caught(monkeypatch):
    """A dropped S^T k term in the p recursion makes the dense-KKT pin fail."""
    qp = W.random_general(0, 3, 2, 6, 4, 2)
    Qh, Rh, Sh, qh, rh = _aug_random(qp, 0.37, 0)
    orig = lq.riccati

    def bad(A, B, c, Qh, Rh, Sh, qh, rh):
        P, p, K, kff, G = orig(A, B, c, Qh, Rh, Sh, qh, rh)
        N = A.shape[0]
        p2 = p.copy()
        for k in range(N - 1, -1, -1):
            p2[k] = qh[k] + A[k].T @ (p2[k + 1] + P[k + 1] @ (B[k] @ kff[k] + c[k]))
        kk = np.stack([-G[k] @ (B[k].T @ (p2[k + 1] + P[k + 1] @ c[k]) + rh[k]) for k in range(N)])
        return P, p2, K, kk, G

    monkeypatch.setattr(lq, "riccati", bad)
    x, u = lq.lq_solve(qp, Qh, Rh, Sh, qh, rh, qp.x0)
    xd, ud, _ = lq.dense_kkt_lq(qp.A, qp.B, qp.c, Qh, Rh, Sh, qh, rh, qp.x0)
    assert not np.allclose(u, ud, atol=1e-6)
