"""GPU parity of the FastSLS duals (sls_tau, App. B) and of the alternation
between the robust controller and the tightened nominal QP (fastsls_solve,
Sec. III-D, eq. nmpc_problem_tightened) against the FP64 oracle
(oracle/fastsls.py).  Tolerances: 1e-10 relative for the FP64 duals from the
same multipliers; 1e-6 relative (FP64 solves to a 1e-10 KKT residual, the
oracle's exact optimum) for the alternation's iterates."""
import dataclasses

import numpy as np
import pytest

from oracle import fastsls, kkt, lq
from oracle import sls as osls
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b))))) if b.size else 0.0


def tight_settings(**kw):
    return native.default_settings(precision=native.GPUSLS_FP64, eps=1e-10, eps_kkt=1e-10, eps_floor=1e-12,
                                   max_iter=200000, **kw)


@pytest.mark.parametrize("seed", [1, 2])
def test_sls_tau_matches_oracle(lib, seed):
    """tau from the GPU's row norms and given multipliers of both signs
    equals the oracle's App. B duals (with the |lambda| reading)."""
    from paper_2604_07644_b300.api import SLS
    qp, sp = W.fastsls_problem(seed)
    s = SLS(sp.nx, sp.nu, sp.N, sp.nc, sp.nf, per_j_tau=True, precision=native.GPUSLS_FP64)
    Px, Pu, h, hf = s.solve(sp)
    lam = np.random.default_rng(seed).standard_normal(qp.m)
    got = s.tau(lam)
    s.close()
    Pxo, Puo, _, _, _ = osls.solve(sp)
    want = fastsls.taus(sp, Pxo, Puo, lam)
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
    assert np.all(got[np.triu_indices(sp.N, 0, sp.N)[0], np.triu_indices(sp.N, 0, sp.N)[1]] == 0.0)


def test_sls_tau_rejects_a_handle_without_a_solve(lib):
    from paper_2604_07644_b300.api import SLS
    s = SLS(3, 2, 5, 3, 2, per_j_tau=True)
    with pytest.raises(RuntimeError):
        s.tau(np.zeros(5 * 3 + 2))
    s.close()


@pytest.mark.parametrize("seed", [1, 3])
def test_alternation_steps_match_oracle(lib, seed):
    """Three RTI-chained calls (one step each, tau_out of a call is tau_in of
    the next) reproduce the oracle's alternation step by step: margins,
    Phi, nominal trajectory and duals."""
    from paper_2604_07644_b300.api import FastSLS
    qp, sp = W.fastsls_problem(seed)
    hist = fastsls.alternation(qp, sp, 3)
    f = FastSLS(qp, sp, tight_settings())
    tau = None
    for i in range(3):
        r = f.step(1, tau_in=tau)
        o = hist[i]
        assert r["info"]["status"] == native.GPUSLS_OK
        assert rel(r["h"], o["h"]) < 1e-9 and rel(r["hf"], o["hf"]) < 1e-9
        assert rel(r["Phix"], o["Phix"]) < 1e-9 and rel(r["Phiu"], o["Phiu"]) < 1e-9
        assert rel(r["x"], o["x"]) < 1e-6 and rel(r["u"], o["u"]) < 1e-6, (i, rel(r["x"], o["x"]))
        assert rel(r["tau"], o["tau"]) < 1e-6, (i, rel(r["tau"], o["tau"]))
        assert kkt.kkt_residual(o["qp"], r["x"], r["u"], r["lam"]) <= 1.0001e-10
        tau = f.tau.clone()
    f.close()


def test_multi_step_call_equals_chained_calls(lib):
    """fastsls_solve with iters = 3 gives what three chained one-step calls
    give (same kernels, same warm ADMM state)."""
    from paper_2604_07644_b300.api import FastSLS
    qp, sp = W.fastsls_problem(2)
    f1 = FastSLS(qp, sp, tight_settings())
    tau = None
    for _ in range(3):
        r1 = f1.step(1, tau_in=tau)
        tau = f1.tau.clone()
    f3 = FastSLS(qp, sp, tight_settings())
    r3 = f3.step(3)
    for k in ("x", "u", "lam", "h", "hf", "tau", "Phix"):
        assert np.array_equal(r1[k], r3[k]), k
    f1.close()
    f3.close()


def _disturbed_violation(qp, r, samples, seed=0):
    g = np.random.default_rng(seed)
    N, nx, nu = qp.N, qp.nx, qp.nu
    worst = -np.inf
    for _ in range(samples):
        w = g.standard_normal((N, nx))
        w /= np.linalg.norm(w, axis=1, keepdims=True)
        X, U = r["x"].copy(), r["u"].copy()
        for k in range(1, N + 1):
            for j in range(k):
                X[k] += r["Phix"][(k - 1) * nx:k * nx, j * nx:(j + 1) * nx] @ w[j]
                if k < N:
                    U[k] += r["Phiu"][k * nu:(k + 1) * nu, j * nx:(j + 1) * nx] @ w[j]
        v = lq.G_apply(qp, X, U)
        worst = max(worst, float(np.max(np.maximum(v - qp.hi, qp.lo - v))))
    return worst


def test_humanoid_75d_step_full_size(lib):
    """One alternation step at the humanoid size (nx=75, nu=21, N=40, FP32
    QP and SLS, the benchmark's launch): the margins match the oracle's SLS
    solve (1e-4 relative), the tightened QP is solved to a 1e-4 KKT residual,
    sampled duals equal App. B's formula on the returned Phi and
    multipliers, and disturbed closed-loop trajectories stay inside the
    original bounds.  A second step from the returned duals converges too."""
    from paper_2604_07644_b300.api import FastSLS
    qp, sp = W.fastsls_problem(0, 75, 21, 40, w_range=(0.001, 0.01), tag=4)
    s = native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, max_iter=6000)
    f = FastSLS(qp, sp, s, sls_precision=native.GPUSLS_FP32)
    r = f.step(1)
    assert r["info"]["status"] == native.GPUSLS_OK
    _, _, h, hf, _ = osls.solve(sp)
    assert rel(r["h"], h) < 1e-4 and rel(r["hf"], hf) < 1e-4
    qt = fastsls.tighten(qp, r["h"], r["hf"])
    assert kkt.kkt_residual(qt, r["x"], r["u"], r["lam"]) <= 1.0001e-4
    N, nc, nx, nu = sp.N, sp.nc, sp.nx, sp.nu
    lam = np.abs(r["lam"])
    for k, j in [(5, 2), (20, 0), (39, 38)]:
        M = sp.C[k] @ r["Phix"][(k - 1) * nx:k * nx, j * nx:(j + 1) * nx] + \
            sp.D[k] @ r["Phiu"][k * nu:(k + 1) * nu, j * nx:(j + 1) * nx]
        want = lam[k * nc:(k + 1) * nc] / np.sqrt(np.sum(M * M, axis=1) + 1e-8)
        assert np.max(np.abs(r["tau"][k, j, :nc] - want)) <= 1e-4 * max(1.0, np.max(want))
    assert _disturbed_violation(qp, r, 10) <= 1e-4
    r2 = f.step(1, tau_in=f.tau.clone())
    assert r2["info"]["status"] == native.GPUSLS_OK
    f.close()
