"""Build the native library libgpusls.so in-tree with nvcc for sm_103a.

Usage: python -m paper_2604_07644_b300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libgpusls.so")
SOURCES = ["qp.cu", "qp_kernel_f32.cu", "qp_kernel_f64.cu", "sls.cu", "mlp.cu", "models.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources() -> list[str]:
    return [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "gpusls.h")]
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object in parallel (the two solve-kernel
    instantiations dominate), then link libgpusls.so."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    with tempfile.TemporaryDirectory() as tmp:
        procs = []
        for src in sources():
            obj = os.path.join(tmp, os.path.basename(src) + ".o")
            procs.append((obj, subprocess.Popen([nvcc, *flags, "-c", "-o", obj, src], stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
        failed = False
        for obj, pr in procs:
            out, _ = pr.communicate()
            if pr.returncode != 0:
                failed = True
                sys.stderr.write(out)
            elif verbose:
                sys.stderr.write(out)
        if failed:
            raise RuntimeError("nvcc failed building libgpusls.so")
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *[o for o, _ in procs]],
                           capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed linking libgpusls.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
