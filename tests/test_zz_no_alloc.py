"""gpusls_kkt_noalloc: the allocation-free KKT residual.

Callers that cannot allocate device memory at the point of use (real-time
loops where cudaMalloc may block, contexts that forbid allocation, runtimes
that own every buffer) call it without a handle; its scratch is a fixed device
array.  This file runs last (pytest collects it after the others) and must
pass both alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi")


def _dev(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def prepare(qp, x, u, lam):
    """Device copies of the problem and the point, and the output buffer."""
    t = {f: _dev(getattr(qp, f)) for f in FIELDS}
    for f in ("C", "D", "CN"):
        if t[f].numel() == 0:
            t[f] = _dev(np.zeros(1))
    t.update(x0=_dev(qp.x0), x=_dev(x), u=_dev(u), lam=_dev(lam),
             out=torch.full((5,), -1.0, dtype=torch.float64, device="cuda"))
    return qp, t


def call(prepared):
    """One gpusls_kkt_noalloc call on prepared device buffers (no torch
    allocation on this path)."""
    qp, t = prepared
    lib = native.load()
    d = native.qp_dims(*qp.dims())
    p = lambda z: ctypes.c_void_p(z.data_ptr())  # noqa: E731
    st = lib.gpusls_kkt_noalloc(d, *[p(t[f]) for f in FIELDS], p(t["x0"]), p(t["x"]), p(t["u"]), p(t["lam"]),
                                p(t["out"]), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    native.check(st, "gpusls_kkt_noalloc")


def noalloc(qp, x, u, lam):
    prepared = prepare(qp, x, u, lam)
    call(prepared)
    torch.cuda.synchronize()
    return prepared[1]["out"].cpu().numpy()


def reference(qp, x, u, lam):
    from paper_2604_07644_b300.api import QPBatch
    b = QPBatch([qp], native.default_settings())
    v = b.kkt([x], [u], [lam])[0]
    b.close()
    return v


def test_noalloc_matches_qp_kkt_on_consecutive_calls(lib):
    """Two calls in a row on different problems (the shared scratch is reused)
    agree with the handle-based qp_kkt."""
    from paper_2604_07644_b300.api import QPBatch
    big = W.quadruped_61d(0)
    b = QPBatch([big], native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5))
    r = b.solve()
    b.close()
    small = W.tiny(2)
    g = np.random.default_rng(0)
    xs = g.standard_normal((small.N + 1, small.nx))
    us = g.standard_normal((small.N, small.nu))
    ls = g.standard_normal(small.m)
    cases = [(big, r.dx[0], r.du[0], r.lam[0]), (small, xs, us, ls), (big, r.dx[0] + 1e-3, r.du[0], r.lam[0])]
    for qp, x, u, lam in cases:
        got = noalloc(qp, x, u, lam)
        ref = reference(qp, x, u, lam)
        assert abs(got[0] - ref) < 1e-12 + 1e-9 * abs(ref), (got, ref)
        assert abs(got[0] - max(got[1:])) == 0.0


def test_noalloc_calls_allocate_no_device_memory(lib):
    """After a first call, further calls change neither the device's free
    memory (cudaMemGetInfo) nor the torch caching allocator's counters."""
    qp = W.quadrotor_12d(0)
    g = np.random.default_rng(1)
    prepared = prepare(qp, g.standard_normal((qp.N + 1, qp.nx)), g.standard_normal((qp.N, qp.nu)),
                       g.standard_normal(qp.m))
    call(prepared)
    first = prepared[1]["out"].clone()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st0 = torch.cuda.memory_stats()
    for _ in range(5):
        call(prepared)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    st1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocated_bytes.all.current", "reserved_bytes.all.current", "num_alloc_retries"):
        assert st1.get(key, 0) == st0.get(key, 0), key
    assert torch.equal(prepared[1]["out"], first)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    lib_ = native.load()
    d = native.qp_dims(80, 64, 2000, 0, 0)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib_.gpusls_kkt_noalloc(d, *([p] * 18), ctypes.c_void_p(0))
    assert st == native.GPUSLS_ERR_INVALID
    assert "exceeds the fixed scratch" in native.last_error()
