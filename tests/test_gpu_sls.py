"""GPU parity of the SLS solve (Phi_x, Phi_u, margins) against the FP64 oracle
(calls through the C ABI).  Tolerances: 1e-6 relative FP64, 1e-4 FP32."""
import numpy as np
import pytest

from oracle import sls as osls
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b))))) if np.size(b) else 0.0


def run(sp, prec):
    from paper_2604_07644_b300.api import SLS
    s = SLS(sp.nx, sp.nu, sp.N, sp.nc, sp.nf, per_j_tau=sp.tau is not None, precision=prec)
    out = s.solve(sp)
    s.close()
    return out


@pytest.mark.parametrize("prec", [native.GPUSLS_FP64, native.GPUSLS_FP32])
@pytest.mark.parametrize("tau_mode", ["zero", "uniform"])
@pytest.mark.parametrize("dims", [(3, 2, 5, 3, 2), (6, 3, 9, 4, 1), (12, 4, 17, 6, 3), (2, 1, 1, 2, 2), (4, 2, 2, 0, 0)])
def test_sls_matches_oracle(lib, dims, tau_mode, prec):
    sp = W.sls_small(1, *dims, tau_mode=tau_mode)
    Phix, Phiu, h, hf = run(sp, prec)
    oPx, oPu, oh, ohf, _ = osls.solve(sp)
    tol = 1e-6 if prec == native.GPUSLS_FP64 else 1e-4
    assert rel(Phix, oPx) < tol, rel(Phix, oPx)
    assert rel(Phiu, oPu) < tol, rel(Phiu, oPu)
    if sp.nc:
        assert rel(h, oh) < tol, rel(h, oh)
    if sp.nf:
        assert rel(hf, ohf) < tol, rel(hf, ohf)
    # causality: strictly upper blocks are exactly zero
    nx, nu, N = sp.nx, sp.nu, sp.N
    for j in range(N):
        for k in range(1, j + 1):
            assert np.all(Phix[(k - 1) * nx:k * nx, j * nx:(j + 1) * nx] == 0)
        for k in range(0, j + 1):
            assert np.all(Phiu[k * nu:(k + 1) * nu, j * nx:(j + 1) * nx] == 0)


@pytest.mark.parametrize("tau_mode", ["zero", "uniform"])
def test_sls_humanoid_75d_full_size(lib, tau_mode):
    """Humanoid-shaped SLS (nx=75, nu=21, N=40, nc=29, nf=8): FP64 Phi and
    margins vs the oracle, FP32 within 1e-4."""
    sp = W.sls_problem(0, tau_mode=tau_mode)
    oPx, oPu, oh, ohf, _ = osls.solve(sp)
    for prec, tol in [(native.GPUSLS_FP64, 1e-6), (native.GPUSLS_FP32, 1e-4)]:
        Phix, Phiu, h, hf = run(sp, prec)
        assert rel(Phix, oPx) < tol and rel(Phiu, oPu) < tol
        assert rel(h, oh) < tol and rel(hf, ohf) < tol
