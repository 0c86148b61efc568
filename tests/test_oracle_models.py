"""Pins of the oracle's analytic models and SQP / RTI loop (App. C, App. D,
Sec. III-B, Sec. IV-C)."""
import numpy as np
import pytest

from oracle import admm, models as M
from paper_2604_07644_b300 import workloads as W

SPECS = [("dubins", lambda: W.dubins(0)), ("quad2d", lambda: W.quad2d(0, N=20))]


def qp_solver(qp):
    return admm.exact_solution(qp, tol=1e-6, max_iter=20000)


def _random_point(m, g):
    x = g.standard_normal(m.nx)
    u = m.uref + g.standard_normal(m.nu)
    return x, u


@pytest.mark.parametrize("name,make", SPECS)
def test_jacobians_match_central_differences(name, make):
    """The hand-derived A = df/dx, B = df/du against central differences of
    the dynamics (an independent route: a wrong sign or a dropped term in
    either fails)."""
    m = make()
    g = np.random.default_rng(1)
    for _ in range(5):
        x, u = _random_point(m, g)
        A, B = M.jacobians(m, x, u)
        h = 1e-6
        Afd = np.stack([(M.dynamics(m, x + h * e, u) - M.dynamics(m, x - h * e, u)) / (2 * h)
                        for e in np.eye(m.nx)], axis=1)
        Bfd = np.stack([(M.dynamics(m, x, u + h * e) - M.dynamics(m, x, u - h * e)) / (2 * h)
                        for e in np.eye(m.nu)], axis=1)
        assert np.allclose(A, Afd, atol=1e-8) and np.allclose(B, Bfd, atol=1e-8)


def test_dynamics_match_the_appendix_formulas():
    """Spot values: the Dubins car moves v dt along its heading and turns by
    omega dt (App. C); the quadrotor at hover thrust stays put, and a thrust
    difference spins it up by L (u2 - u1) / J dt (App. D)."""
    m = W.dubins(0)
    y = M.dynamics(m, np.array([1.0, 2.0, np.pi / 2]), np.array([0.5]))
    assert np.allclose(y, [1.0, 2.0 + m.v * m.dt, np.pi / 2 + 0.5 * m.dt], atol=1e-15)
    q = W.quad2d(0)
    uh = q.mass * q.grav / 2.0
    assert np.allclose(M.dynamics(q, np.zeros(6), np.array([uh, uh])), 0.0, atol=1e-14)
    y = M.dynamics(q, np.zeros(6), np.array([uh - 1.0, uh + 1.0]))
    assert np.isclose(y[5], q.dt * q.arm * 2.0 / q.inertia) and abs(y[4]) < 1e-14


@pytest.mark.parametrize("name,make", SPECS)
def test_linearization_is_first_order_accurate(name, make):
    """The LTV-QP predicts the nonlinear dynamics and obstacle constraints to
    second order: halving a perturbation quarters the prediction error."""
    m = make()
    g = np.random.default_rng(2)
    X, U = m.initial_guess()
    X = X + 0.1 * g.standard_normal(X.shape)
    U = U + 0.1 * g.standard_normal(U.shape)
    qp = M.linearize(m, X, U, m.x0)
    dX = g.standard_normal(X.shape)
    dU = g.standard_normal(U.shape)
    errs = []
    for t in (1e-2, 5e-3):
        k = 3
        pred = X[k + 1] + qp.A[k] @ (t * dX[k]) + qp.B[k] @ (t * dU[k]) + qp.c[k] + (t * dX[k + 1]) * 0.0
        true = M.dynamics(m, X[k] + t * dX[k], U[k] + t * dU[k])
        gpred = M.obstacle_g(m, X[k]) + qp.C[k, m.nu:] @ (t * dX[k])
        gtrue = M.obstacle_g(m, X[k] + t * dX[k])
        errs.append((np.max(np.abs(pred - true)), np.max(np.abs(gpred - gtrue))))
    for i in range(2):
        assert errs[1][i] < 0.3 * errs[0][i] + 1e-15
    # bounds in deviation form: u_lo <= u_k + du_k <= u_hi
    nc = m.nu + m.n_obs
    assert np.allclose(qp.hi[2 * nc:2 * nc + m.nu], m.u_hi - U[2])
    assert np.allclose(qp.x0, m.x0 - X[0])


@pytest.mark.parametrize("name,make", SPECS)
def test_sqp_converges_to_a_feasible_stationary_point(name, make):
    """SQP iterations shrink the step and the infeasibility (Gauss-Newton
    SQP converges linearly: 8 iterations take the step below 1 % of the
    first); the accepted step sizes lower the merit."""
    m = make()
    X, U = m.initial_guess()
    hist = M.sqp(m, X, U, m.x0, 8, qp_solver)
    steps = [np.max(np.abs(h[3])) for h in hist]
    assert steps[-1] < 1e-2 * steps[0]
    Xf, Uf = hist[-1][0], hist[-1][1]
    assert M.infeasibility(m, Xf, Uf, m.x0) < 1e-3 * M.infeasibility(m, hist[0][0], hist[0][1], m.x0) + 1e-9
    prev = M.merit(m, X, U, m.x0, 100.0)
    for Xi, Ui, a, dx, du in hist:
        cur = M.merit(m, Xi, Ui, m.x0, 100.0)
        assert cur < prev + 1e-9
        prev = cur


def test_rti_from_the_optimum_without_disturbance_follows_the_nominal():
    """A converged SQP nominal is (nearly) a fixed point of RTI: the first
    applied input is u_0 and the next state x_1, up to the size of the last
    SQP step (Gauss-Newton SQP converges linearly)."""
    m = W.dubins(1)
    X, U = m.initial_guess()
    hist = M.sqp(m, X, U, m.x0, 12, qp_solver)
    Xs, Us = hist[-1][:2]
    last = max(np.max(np.abs(hist[-1][3])), np.max(np.abs(hist[-1][4])))
    xs, us, _ = M.rti_rollout(m, Xs, Us, m.x0, np.zeros((1, m.nx)), qp_solver)
    assert np.max(np.abs(us[0] - Us[0])) <= 10 * last + 1e-6
    assert np.max(np.abs(xs[1] - Xs[1])) <= 10 * last + 1e-6


def test_robust_rti_keeps_disturbed_rollouts_out_of_the_obstacles():
    """The robust RTI loop (SLS tightening each step) keeps every disturbed
    closed-loop state of the planar quadrotor outside the obstacle on
    sampled disturbances, with nonzero margins."""
    m = W.quad2d(0, N=20)
    X, U = m.initial_guess()
    Xs, Us = M.sqp(m, X, U, m.x0, 6, qp_solver)[-1][:2]
    Wd = W.disturbances(0, 10, 2, m.nx)
    for b in range(2):
        xs, us, hs = M.rti_rollout_robust(m, Xs, Us, m.x0, Wd[:, b], qp_solver)
        assert max(np.max(M.obstacle_g(m, x)) for x in xs) <= 1e-9
        assert max(np.max(h[0]) for h in hs) > 0.0
