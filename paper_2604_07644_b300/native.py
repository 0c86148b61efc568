"""ctypes binding of libgpusls.so (include/gpusls.h): argument marshalling only.

Every compute step runs inside the library's CUDA kernels.  The library must
be built in-tree (python -m paper_2604_07644_b300.build); a missing library
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgpusls.so")

GPUSLS_OK = 0
GPUSLS_MAX_ITER = 1
GPUSLS_ERR_INVALID = -1
GPUSLS_ERR_NOT_SPD = -2
GPUSLS_ERR_NAN = -3
GPUSLS_ERR_INFEASIBLE = -4
GPUSLS_ERR_CUDA = -5
GPUSLS_ERR_TIMEOUT = -6
GPUSLS_FP64 = 0
GPUSLS_FP32 = 1
GPUSLS_TF32 = 2
GPUSLS_MIXED = 3
GPUSLS_FEATURE_P = 16

STATUS_NAMES = {0: "ok", 1: "max_iter", -1: "invalid", -2: "not_spd", -3: "nan", -4: "infeasible",
                -5: "cuda", -6: "timeout"}


class qp_dims(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nu", C.c_int32), ("N", C.c_int32), ("nc", C.c_int32), ("nf", C.c_int32)]


class qp_settings(C.Structure):
    _fields_ = [("rho0", C.c_double), ("eps", C.c_double), ("eps_kkt", C.c_double), ("rho_min", C.c_double),
                ("rho_max", C.c_double), ("sigma", C.c_int32), ("check_every", C.c_int32),
                ("max_iter", C.c_int32), ("precision", C.c_int32), ("cluster", C.c_int32),
                ("fixed_iters", C.c_int32), ("max_refine", C.c_int32), ("fallback_iters", C.c_int32),
                ("occupancy", C.c_int32), ("eps_floor", C.c_double), ("schedule", C.c_int32),
                ("factorization", C.c_int32)]


class qp_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("refactors", C.c_int32), ("refines", C.c_int32),
                ("fallback", C.c_int32), ("pad", C.c_int32),
                ("rho", C.c_double), ("r_prim", C.c_double), ("r_dual", C.c_double), ("kkt", C.c_double)]


GPUSLS_MODEL_DUBINS = 0
GPUSLS_MODEL_QUAD2D = 1
GPUSLS_MODEL_MAX_OBS = 16


class model_spec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("N", C.c_int32), ("n_obs", C.c_int32), ("pad", C.c_int32),
                ("dt", C.c_double), ("v", C.c_double), ("mass", C.c_double), ("grav", C.c_double),
                ("arm", C.c_double), ("inertia", C.c_double), ("u_lo", C.c_double * 2), ("u_hi", C.c_double * 2),
                ("xref", C.c_double * 6), ("uref", C.c_double * 2), ("Qd", C.c_double * 6), ("Rd", C.c_double * 2),
                ("QNd", C.c_double * 6), ("E", C.c_double * 36), ("obs", C.c_double * (3 * GPUSLS_MODEL_MAX_OBS))]


P = C.c_void_p
DP = C.c_void_p   # device pointer to double

# name -> (restype, argtypes); the exported symbols of include/gpusls.h
SIGNATURES = {
    "qp_default_settings": (None, [C.POINTER(qp_settings)]),
    "gpusls_last_error": (C.c_char_p, []),
    "qp_setup": (C.c_int, [C.POINTER(P), qp_dims, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP,
                           C.c_double, C.POINTER(qp_settings), P]),
    "qp_batch_setup": (C.c_int, [C.POINTER(P), C.c_int32, C.POINTER(qp_dims), DP, DP, DP, DP, DP, DP, DP, DP,
                                 DP, DP, DP, DP, DP, C.POINTER(C.c_double), C.POINTER(qp_settings), P]),
    "qp_solve": (C.c_int, [P, DP, C.c_int32, C.c_double, DP, DP, DP, C.POINTER(qp_info)]),
    "qp_set_warm_start": (C.c_int, [P, DP, DP, C.POINTER(C.c_double)]),
    "qp_get_state": (C.c_int, [P, DP, DP, C.POINTER(C.c_double)]),
    "qp_update": (C.c_int, [P, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP]),
    "qp_reset": (C.c_int, [P]),
    "qp_kkt": (C.c_int, [P, DP, DP, DP, DP, C.POINTER(C.c_double)]),
    "qp_riccati": (C.c_int, [P, DP, DP]),
    "qp_destroy": (None, [P]),
    "sls_setup": (C.c_int, [C.POINTER(P), qp_dims, C.c_int32, C.c_int32, P]),
    "sls_setup_ex": (C.c_int, [C.POINTER(P), qp_dims, C.c_int32, C.c_int32, C.POINTER(qp_settings), P]),
    "sls_solve": (C.c_int, [P, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP, DP]),
    "sls_destroy": (None, [P]),
    "sls_tau": (C.c_int, [P, DP, C.c_double, DP]),
    "fastsls_solve": (C.c_int, [P, P] + [DP] * 12 + [C.c_int32, C.c_double] + [DP] * 9 + [C.POINTER(qp_info)]),
    "mlp_create": (C.c_int, [C.POINTER(P), C.c_int32, C.c_int32, C.c_int32, C.c_int32, P]),
    "mlp_set_params": (C.c_int, [P, DP, DP, DP, DP, DP, DP]),
    "mlp_get_params": (C.c_int, [P, DP, DP, DP, DP, DP, DP]),
    "mlp_fit_normalization": (C.c_int, [P, DP, DP, C.c_int32]),
    "mlp_forward": (C.c_int, [P, DP, C.c_int32, DP]),
    "mlp_set_normalization": (C.c_int, [P, DP, DP, DP, DP]),
    "mlp_get_normalization": (C.c_int, [P, DP, DP, DP, DP]),
    "mlp_save": (C.c_int, [P, C.c_char_p]),
    "mlp_load": (C.c_int, [P, C.c_char_p]),
    "mlp_gradients": (C.c_int, [P, DP, DP, C.c_int32, DP, C.POINTER(C.c_float)]),
    "mlp_train_step": (C.c_int, [P, DP, DP, C.c_int32, C.c_float, C.POINTER(C.c_float)]),
    "mlp_destroy": (None, [P]),
    "qp_warm_start_mlp": (C.c_int, [P, P, DP, C.c_double, C.c_double]),
    "qp_graph_create": (C.c_int, [C.POINTER(P), P, P, DP, DP, DP, DP, DP, DP, DP, C.c_double, C.c_double]),
    "qp_graph_launch": (C.c_int, [P, P]),
    "qp_graph_destroy": (None, [P]),
    "qp_graph_kernel_count": (C.c_int, [P, C.POINTER(C.c_int32)]),
    "qp_features": (C.c_int, [P, DP, P, C.c_int32, C.c_int32, P]),
    "qp_warm_start_heads": (C.c_int, [P, C.c_int32, C.POINTER(P), C.POINTER(P), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int32), DP, C.c_double, C.c_double]),
    "qp_graph_create_heads": (C.c_int, [C.POINTER(P), P, C.c_int32, C.POINTER(P), C.POINTER(P),
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32), DP, DP, DP, DP, P, DP,
                                        C.c_double, C.c_double]),
    "model_dims": (C.c_int, [C.POINTER(model_spec), C.POINTER(qp_dims)]),
    "model_linearize": (C.c_int, [C.POINTER(model_spec), C.c_int32] + [DP] * 17 + [P]),
    "model_merit": (C.c_int, [C.POINTER(model_spec), C.c_int32] + [DP] * 6 + [C.c_double, DP, P]),
    "sqp_setup": (C.c_int, [C.POINTER(P), C.POINTER(model_spec), C.c_int32, C.POINTER(qp_settings), C.c_int32, P]),
    "sqp_solve": (C.c_int, [P, DP, DP, DP, C.c_int32, C.c_double, C.c_int32, C.POINTER(C.c_double),
                            C.POINTER(qp_info)]),
    "rti_step": (C.c_int, [P] + [DP] * 7 + [C.POINTER(qp_info)]),
    "sqp_reset_duals": (C.c_int, [P]),
    "sqp_destroy": (None, [P]),
    "gpusls_kkt_noalloc": (C.c_int, [qp_dims] + [DP] * 18 + [P]),
}

_lock = threading.Lock()
_lib = None


def header_symbols() -> list[str]:
    """Function names declared in include/gpusls.h."""
    import re
    hdr = os.path.join(os.path.dirname(_PKG), "include", "gpusls.h")
    txt = open(hdr).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted({n for n in names if n not in ("if", "while", "for", "return", "sizeof")})


def load(path: str = LIB_PATH):
    """Load the library (once) and declare the signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libgpusls.so not built ({path}); run python -m paper_2604_07644_b300.build")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            if hasattr(lib, name):
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
        _lib = lib
        return lib


def last_error() -> str:
    return load().gpusls_last_error().decode()


def check(status: int, what: str):
    if status < 0:
        raise RuntimeError(f"{what} failed with {STATUS_NAMES.get(status, status)}: {last_error()}")
    return status


def default_settings(**kw) -> qp_settings:
    s = qp_settings()
    load().qp_default_settings(C.byref(s))
    for k, v in kw.items():
        if not hasattr(s, k):
            raise KeyError(k)
        setattr(s, k, v)
    return s
