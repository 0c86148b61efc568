"""Edge cases of the LTV-QP path against the FP64 oracle: degenerate sizes
(a single stage, one state, one input, no constraint rows), the largest
sizes a CTA's shared memory accepts, problems too large for it (rejected
with GPUSLS_ERR_INVALID, after which the library keeps working), ragged
batches mixing all of these, and primal-infeasible QPs (classified
GPUSLS_ERR_INFEASIBLE at max_iter as the oracle classifies them, with finite
outputs)."""
import numpy as np
import pytest

from oracle import admm
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {native.GPUSLS_FP64: 1e-9, native.GPUSLS_FP32: 1e-4}


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b))))) if b.size else 0.0


def fixed(qps, prec, cluster, iters=5, rho=0.3):
    from paper_2604_07644_b300.api import QPBatch
    b = QPBatch(qps, native.default_settings(precision=prec, cluster=cluster, sigma=0, fixed_iters=iters), rho=rho)
    r = b.solve()
    b.close()
    return r


DEGENERATE = [(1, 1, 1, 0, 0), (1, 1, 1, 1, 1), (3, 1, 1, 2, 1), (2, 1, 2, 0, 2), (5, 2, 3, 4, 0)]
LARGEST = [(80, 32, 3, 32, 16), (80, 32, 5, 16, 8), (64, 32, 4, 64, 64)]


@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32])
@pytest.mark.parametrize("dims", DEGENERATE + LARGEST)
def test_sizes_match_oracle(lib, dims, prec):
    qp = W.random_general(9, *dims)
    o = admm.admm(qp, admm.Settings(rho0=0.3, sigma=0), iters=5)
    for cs in (1, 4, 8):
        r = fixed([qp], prec, cs)
        assert rel(r.dx[0], o.x) < TOL[prec] and rel(r.du[0], o.u) < TOL[prec], (cs, rel(r.dx[0], o.x))
        assert rel(r.lam[0], o.lam) < TOL[prec]


def test_oversized_problem_is_rejected_and_the_library_keeps_working(lib):
    """nx = 80, nu = 32 with 64 stage and 64 terminal rows: the FP64 shared-
    memory layout does not fit a CTA, so setup returns GPUSLS_ERR_INVALID;
    the FP32 one either fits (and matches the oracle) or is rejected the same
    way at every cluster size -- never a CUDA error -- and a normal problem
    solves correctly afterwards."""
    from paper_2604_07644_b300.api import QPBatch
    qp = W.random_general(9, 80, 32, 3, 64, 64)
    with pytest.raises(RuntimeError, match="invalid"):
        QPBatch([qp], native.default_settings(precision=native.GPUSLS_FP64))
    o = admm.admm(qp, admm.Settings(rho0=0.3, sigma=0), iters=5)
    for cs in (1, 4, 8):
        try:
            r = fixed([qp], native.GPUSLS_FP32, cs)
        except RuntimeError as e:
            assert "invalid" in str(e), str(e)
            continue
        assert rel(r.dx[0], o.x) < 1e-4
    small = W.plain_4d(0)
    o2 = admm.admm(small, admm.Settings(rho0=0.3, sigma=0), iters=5)
    r = fixed([small], native.GPUSLS_FP64, 2)
    assert rel(r.dx[0], o2.x) < 1e-9


def test_ragged_batch_with_degenerate_members(lib):
    """One launch over a single-stage QP, a QP without constraint rows, a
    one-state QP and a 64-stage quadrotor-shaped QP gives each its own
    oracle iterates."""
    qps = [W.random_general(3, 1, 1, 1, 1, 1), W.random_general(4, 6, 2, 9, 0, 0), W.random_general(5, 1, 1, 7, 2, 1),
           W.quadrotor_12d(2)]
    r = fixed(qps, native.GPUSLS_FP64, 4)
    for i, qp in enumerate(qps):
        o = admm.admm(qp, admm.Settings(rho0=0.3, sigma=0), iters=5)
        assert rel(r.dx[i], o.x) < 1e-9 and rel(r.lam[i], o.lam) < 1e-9, i


def test_infeasible_qp_is_classified_at_max_iter(lib):
    """x0 outside the state bound |x| <= 5 of stage 0 (x_0 = x0 is fixed):
    no feasible point exists; the solve stops at max_iter, its status is
    GPUSLS_ERR_INFEASIBLE (the certificate holds), the call returns
    GPUSLS_MAX_ITER, the outputs are finite with a primal residual that
    stays large, and the other QP of the batch still converges."""
    from paper_2604_07644_b300.api import QPBatch
    bad = W.plain_4d(0)
    bad.x0 = bad.x0.copy()
    bad.x0[0] = 9.0
    good = W.plain_4d(1)
    b = QPBatch([bad, good], native.default_settings(precision=native.GPUSLS_FP64, max_iter=600))
    r = b.solve()
    b.close()
    assert r.status == native.GPUSLS_MAX_ITER
    assert r.info[0]["status"] == native.GPUSLS_ERR_INFEASIBLE and r.info[0]["r_prim"] > 1.0
    assert all(np.isfinite(a).all() for a in (r.dx[0], r.du[0], r.lam[0]))
    assert r.info[1]["status"] == native.GPUSLS_OK


@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32])
@pytest.mark.parametrize("case", ["x0_outside_the_box", "unreachable_terminal_box", "feasible_cut_short"])
def test_max_iter_classification_matches_oracle(lib, case, prec):
    """The certificate at max_iter (Farkas, from the multipliers' change
    over the last check interval) classifies as the oracle's ADMM does:
    infeasible by construction -> GPUSLS_ERR_INFEASIBLE, a feasible QP cut
    short -> GPUSLS_MAX_ITER."""
    from paper_2604_07644_b300.api import QPBatch
    qp, it = {"x0_outside_the_box": (W.infeasible_x0(), 600),
              "unreachable_terminal_box": (W.infeasible_terminal(), 600),
              "feasible_cut_short": (W.plain_4d(0), 20)}[case]
    o = admm.admm(qp, admm.Settings(max_iter=it))
    b = QPBatch([qp], native.default_settings(precision=prec, max_iter=it, eps_kkt=0.0))
    r = b.solve()
    b.close()
    want = native.GPUSLS_ERR_INFEASIBLE if o.infeasible else native.GPUSLS_MAX_ITER
    assert r.info[0]["status"] == want, (r.info[0], o.infeasible)
    assert (case != "feasible_cut_short") == o.infeasible


@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32])
def test_nan_in_the_data_is_reported_and_the_library_keeps_working(lib, prec):
    """A NaN injected on the host into q makes the iterates NaN: the first
    check reports GPUSLS_ERR_NAN (a NaN primal residual is not dropped by
    the max), and a clean QP solves afterwards."""
    import dataclasses

    from paper_2604_07644_b300.api import QPBatch
    qp = W.plain_4d(0)
    q = qp.q.copy()
    q[3, 1] = np.nan
    bad = dataclasses.replace(qp, q=q)
    s = native.default_settings(precision=prec, max_iter=200)
    b = QPBatch([bad], s)
    with pytest.raises(RuntimeError, match="failed with nan"):
        b.solve()
    b.close()
    b = QPBatch([qp], s)
    r = b.solve()
    b.close()
    assert r.info[0]["status"] == native.GPUSLS_OK


@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32, native.GPUSLS_MIXED])
def test_indefinite_input_cost_is_reported_not_spd(lib, prec):
    """R = -I (host-side corrupt cost): R^ = R + rho D^T D is not positive
    definite; the factorization reports GPUSLS_ERR_NOT_SPD (in GPUSLS_MIXED
    through the refined node solve's failed FP32 pivot and its FP64
    elimination)."""
    import dataclasses

    from paper_2604_07644_b300.api import QPBatch
    qp = W.plain_4d(0)
    bad = dataclasses.replace(qp, R=-np.ones_like(qp.R) * np.eye(qp.nu))
    b = QPBatch([bad], native.default_settings(precision=prec))
    with pytest.raises(RuntimeError, match="failed with not_spd"):
        b.solve()
    b.close()


def test_bounded_wait_gives_up_with_timeout_status(lib, monkeypatch):
    """The test hook GPUSLS_TEST_WAIT_TIMEOUT makes every solve wait once
    (bounded) on a copy barrier that nothing completes: the wait gives up,
    the solve reports GPUSLS_ERR_TIMEOUT, and the context stays usable (a
    later solve without the hook converges)."""
    import torch

    from paper_2604_07644_b300.api import QPBatch
    qp = W.plain_4d(0)
    s = native.default_settings(precision=native.GPUSLS_FP32, max_iter=200)
    monkeypatch.setenv("GPUSLS_TEST_WAIT_TIMEOUT", "1")
    b = QPBatch([qp], s)
    with pytest.raises(RuntimeError, match="failed with timeout"):
        b.solve()
    b.close()
    monkeypatch.delenv("GPUSLS_TEST_WAIT_TIMEOUT")
    torch.cuda.synchronize()
    b = QPBatch([qp], s)
    r = b.solve()
    b.close()
    assert r.info[0]["status"] == native.GPUSLS_OK
