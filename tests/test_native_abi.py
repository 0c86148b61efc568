"""The C-ABI library builds for sm_103a, loads, and exports every symbol
declared in include/gpusls.h (no compute calls: runs without a GPU)."""
import ctypes
import os
import subprocess

import pytest

from paper_2604_07644_b300 import build, native


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_library_loads_and_exports_header_symbols(libpath):
    lib = ctypes.CDLL(libpath)
    names = native.header_symbols()
    assert "qp_setup" in names and "qp_solve" in names and "sls_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared in gpusls.h but not exported: {missing}"


def test_binding_declares_every_header_symbol():
    names = set(native.header_symbols())
    assert names <= set(native.SIGNATURES), sorted(names - set(native.SIGNATURES))


def test_default_settings_without_gpu(libpath):
    s = native.default_settings()
    assert s.rho0 == 0.1 and s.sigma == 25 and s.check_every == 5 and s.eps == 1e-4


def test_default_settings_fill_every_field(libpath):
    """qp_default_settings writes every field, whatever the struct held."""
    s = native.qp_settings()
    ctypes.memset(ctypes.byref(s), 0xA5, ctypes.sizeof(s))
    native.load().qp_default_settings(ctypes.byref(s))
    assert s.occupancy == 0 and s.schedule == 0 and s.factorization == 0 and s.eps_floor == 0.0
    assert s.cluster == 0 and s.fixed_iters == 0 and s.fallback_iters == 0


def test_invalid_arguments_are_rejected_without_gpu(libpath):
    lib = native.load()
    h = ctypes.c_void_p()
    d = native.qp_dims(0, 1, 1, 0, 0)
    s = native.default_settings()
    st = lib.qp_setup(ctypes.byref(h), d, None, None, None, None, None, None, None, None, None, None, None,
                      None, None, 0.1, ctypes.byref(s), None)
    assert st == native.GPUSLS_ERR_INVALID
    assert "null" in native.last_error() or "dims" in native.last_error()


def test_kernels_are_compiled_for_sm103a(libpath):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout
