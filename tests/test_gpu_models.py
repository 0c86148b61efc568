"""GPU parity of the analytic models and the SQP / RTI outer loop (App. C,
App. D, Sec. III-B, Sec. IV-C) against the FP64 oracle (oracle/models.py):
the parallel linearization and the merit to 1e-12, SQP iterates and step
sizes, classical and robust RTI closed loops under the same disturbances to
1e-6 (the inner QPs solved to a 1e-10 KKT residual on the GPU and exactly by
the oracle)."""
import numpy as np
import pytest
import torch

from oracle import admm, models as M
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu

SPECS = [("dubins", lambda: W.dubins(0)), ("quad2d", lambda: W.quad2d(0, N=20))]
KEYS = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi")


def oracle_qp(qp):
    return admm.exact_solution(qp, tol=1e-6, max_iter=20000)


def tight():
    return native.default_settings(precision=native.GPUSLS_FP64, eps=1e-10, eps_kkt=1e-10, eps_floor=1e-12,
                                   max_iter=200000)


def perturbed_nominals(m, count, seed):
    g = np.random.default_rng(seed)
    X0, U0 = m.initial_guess()
    Xs = np.stack([X0 + 0.2 * g.standard_normal(X0.shape) for _ in range(count)])
    Us = np.stack([U0 + 0.2 * g.standard_normal(U0.shape) for _ in range(count)])
    x0 = np.stack([m.x0 + 0.1 * g.standard_normal(m.nx) for _ in range(count)])
    return Xs, Us, x0


@pytest.mark.parametrize("name,make", SPECS)
def test_linearization_matches_oracle(lib, name, make):
    from paper_2604_07644_b300.api import linearize
    m = make()
    Xs, Us, x0 = perturbed_nominals(m, 3, 1)
    got = linearize(m, Xs, Us, x0)
    for b in range(3):
        o = M.linearize(m, Xs[b], Us[b], x0[b])
        for k in KEYS:
            a, e = got[b][k], getattr(o, k)
            assert np.array_equal(np.isinf(a), np.isinf(e)), k
            fin = np.isfinite(e)
            assert np.max(np.abs(a[fin] - e[fin]), initial=0.0) <= 1e-13 * max(1.0, np.max(np.abs(e[fin]))), k
        assert np.max(np.abs(got[b]["dx0"] - o.x0)) <= 1e-15


@pytest.mark.parametrize("name,make", SPECS)
def test_merit_matches_oracle(lib, name, make):
    import ctypes as C

    from paper_2604_07644_b300.api import _dev64, _dptr, model_spec
    m = make()
    Xs, Us, x0 = perturbed_nominals(m, 2, 2)
    g = np.random.default_rng(3)
    dX, dU = g.standard_normal(Xs.shape), g.standard_normal(Us.shape)
    spec = model_spec(m)
    lib_ = native.load()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    t = [_dev64(v, "cuda") for v in (Xs, Us, dX, dU, x0)]   # kept alive across the calls
    for a in (0.0, 0.5, 1.0):
        alpha = torch.full((2,), a, dtype=torch.float64, device="cuda")
        native.check(lib_.model_merit(C.byref(spec), 2, _dptr(t[0]), _dptr(t[1]), _dptr(t[2]), _dptr(t[3]),
                                      _dptr(alpha), _dptr(t[4]), 100.0, _dptr(out), None), "model_merit")
        got = out.cpu().numpy()
        for b in range(2):
            want = M.merit(m, Xs[b] + a * dX[b], Us[b] + a * dU[b], x0[b], 100.0)
            assert abs(got[b] - want) <= 1e-12 * abs(want)


def test_sqp_matches_oracle_batched(lib):
    """Two Dubins instances in one batch: four SQP iterations (one call per
    iteration) match the oracle's iterates and step sizes."""
    from paper_2604_07644_b300.api import SQP
    ms = [W.dubins(0), W.dubins(1)]
    sq = SQP(ms[0], 2, tight())
    # both trajectories use model 0's data (one spec per handle); instance 1
    # differs in its initial state and nominal
    X0, U0 = ms[0].initial_guess()
    Xs = np.stack([X0, X0 + 0.05])
    Us = np.stack([U0, U0 + 0.1])
    x0 = np.stack([ms[0].x0, ms[0].x0 + np.array([0.0, 0.05, 0.02])])
    sq.set_nominal(Xs, Us)
    sq.set_state(x0)
    hist = [M.sqp(ms[0], Xs[b], Us[b], x0[b], 4, oracle_qp) for b in range(2)]
    for it in range(4):
        a, info = sq.solve(1)
        X = sq.X.cpu().numpy()
        U = sq.U.cpu().numpy()
        for b in range(2):
            Xo, Uo, ao, _, _ = hist[b][it]
            assert a[0, b] == ao, (it, b, a[0, b], ao)
            assert np.max(np.abs(X[b] - Xo)) < 1e-6 and np.max(np.abs(U[b] - Uo)) < 1e-6, (it, b)
    sq.close()


def test_sqp_matches_oracle_quadrotor(lib):
    from paper_2604_07644_b300.api import SQP
    m = W.quad2d(0, N=20)
    sq = SQP(m, 1, tight())
    X0, U0 = m.initial_guess()
    sq.set_nominal(X0[None], U0[None])
    sq.set_state(m.x0[None])
    hist = M.sqp(m, X0, U0, m.x0, 4, oracle_qp)
    for it in range(4):
        a, info = sq.solve(1)
        Xo, Uo, ao, _, _ = hist[it]
        assert a[0, 0] == ao
        assert np.max(np.abs(sq.X.cpu().numpy()[0] - Xo)) < 1e-6
        assert np.max(np.abs(sq.U.cpu().numpy()[0] - Uo)) < 1e-6 * max(1.0, np.max(np.abs(Uo)))
    sq.close()


def test_rti_closed_loop_matches_oracle(lib):
    """Three disturbed closed loops (classical RTI, one batch) from the SQP
    nominal: the visited states and applied inputs match the oracle's."""
    from paper_2604_07644_b300.api import SQP
    m = W.dubins(1)
    X0, U0 = m.initial_guess()
    Xs, Us = M.sqp(m, X0, U0, m.x0, 6, oracle_qp)[-1][:2]
    steps, B = 6, 3
    Wd = W.disturbances(1, steps, B, m.nx)
    sq = SQP(m, B, tight())
    sq.set_nominal(np.repeat(Xs[None], B, 0), np.repeat(Us[None], B, 0))
    sq.set_state(np.repeat(m.x0[None], B, 0))
    xs_g = [sq.x.cpu().numpy().copy()]
    us_g = []
    for t in range(steps):
        sq.rti_step(Wd[t])
        xs_g.append(sq.x.cpu().numpy().copy())
        us_g.append(sq.u0.cpu().numpy().copy())
    for b in range(B):
        xs, us, _ = M.rti_rollout(m, Xs, Us, m.x0, Wd[:, b], oracle_qp)
        assert np.max(np.abs(np.array([x[b] for x in xs_g]) - xs)) < 1e-6
        assert np.max(np.abs(np.array([u[b] for u in us_g]) - us)) < 1e-6
    sq.close()


def test_robust_rti_matches_oracle_and_stays_safe(lib):
    """Robust RTI on the planar quadrotor (controller update from the
    previous duals, SLS tightening, tightened QP each step): states, inputs
    and margins match the oracle's robust loop, and no disturbed state
    enters the obstacle."""
    from paper_2604_07644_b300.api import SQP
    m = W.quad2d(0, N=20)
    X0, U0 = m.initial_guess()
    Xs, Us = M.sqp(m, X0, U0, m.x0, 6, oracle_qp)[-1][:2]
    steps = 5
    Wd = W.disturbances(2, steps, 1, m.nx)
    xs, us, hs = M.rti_rollout_robust(m, Xs, Us, m.x0, Wd[:, 0], oracle_qp)
    sq = SQP(m, 1, tight(), robust=True)
    sq.set_nominal(Xs[None], Us[None])
    sq.set_state(m.x0[None])
    nc = m.nu + m.n_obs
    for t in range(steps):
        sq.rti_step(Wd[t])
        assert np.max(np.abs(sq.x.cpu().numpy()[0] - xs[t + 1])) < 1e-6, t
        assert np.max(np.abs(sq.u0.cpu().numpy()[0] - us[t])) < 1e-6 * max(1.0, np.max(np.abs(us[t])))
        h = sq.hk.cpu().numpy()[:m.N * nc].reshape(m.N, nc)
        assert np.max(np.abs(h - hs[t][0])) < 1e-9 * max(1.0, np.max(np.abs(hs[t][0])))
    assert max(np.max(M.obstacle_g(m, x)) for x in xs) <= 0.0
    sq.close()
