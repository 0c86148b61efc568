"""Python front end of the GPU-SLS library: packs problem data into device
pools (torch tensors, float64) and calls the C ABI.  No arithmetic of the
method happens here.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import os

import numpy as np
import torch

from . import native

QP_FIELDS = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN")


def _dptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_ptr(stream: torch.cuda.Stream | None):
    s = stream or torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def pool(arrays: list[np.ndarray], device="cuda") -> torch.Tensor:
    """Concatenate per-QP arrays (flattened, float64) into one device pool."""
    flat = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in arrays]
    host = np.concatenate(flat) if flat else np.zeros(0)
    if host.size == 0:
        host = np.zeros(1)
    return torch.from_numpy(host).to(device)


@dataclass
class Result:
    dx: list
    du: list
    lam: list
    info: list
    status: int


class QPBatch:
    """A handle over one or more LTV-QPs (qp_batch_setup)."""

    def __init__(self, qps, settings: native.qp_settings | None = None, rho=None, stream=None, device="cuda",
                 pools: dict | None = None):
        self.lib = native.load()
        self.qps = list(qps)
        self.B = len(self.qps)
        self.device = device
        self.stream = stream
        self.settings = settings or native.default_settings()
        dims = (native.qp_dims * self.B)()
        for i, qp in enumerate(self.qps):
            dims[i].nx, dims[i].nu, dims[i].N, dims[i].nc, dims[i].nf = qp.dims()
        self.dims = dims
        if pools is not None:          # device pools of another handle over the same QPs (copied at setup)
            self.pools = pools
        else:
            self.pools = {f: pool([getattr(qp, f) for qp in self.qps], device) for f in QP_FIELDS}
            self.pools["lo"] = pool([qp.lo for qp in self.qps], device)
            self.pools["hi"] = pool([qp.hi for qp in self.qps], device)
        rho_arr = None
        if rho is not None:
            rho_arr = (C.c_double * self.B)(*([float(rho)] * self.B if np.isscalar(rho) else [float(v) for v in rho]))
        h = C.c_void_p()
        p = self.pools
        st = self.lib.qp_batch_setup(C.byref(h), self.B, dims, _dptr(p["A"]), _dptr(p["B"]), _dptr(p["c"]),
                                     _dptr(p["Q"]), _dptr(p["R"]), _dptr(p["S"]), _dptr(p["q"]), _dptr(p["r"]),
                                     _dptr(p["C"]), _dptr(p["D"]), _dptr(p["CN"]), _dptr(p["lo"]), _dptr(p["hi"]),
                                     rho_arr, C.byref(self.settings), _stream_ptr(stream))
        native.check(st, "qp_batch_setup")
        self.h = h
        self.nx = [qp.nx for qp in self.qps]
        self.sizes = dict(
            x=[(qp.N + 1) * qp.nx for qp in self.qps],
            u=[qp.N * qp.nu for qp in self.qps],
            m=[qp.m for qp in self.qps],
            P=[(qp.N + 1) * qp.nx * qp.nx for qp in self.qps],
            K=[qp.N * qp.nu * qp.nx for qp in self.qps],
        )
        self.out_x = torch.zeros(max(1, sum(self.sizes["x"])), dtype=torch.float64, device=device)
        self.out_u = torch.zeros(max(1, sum(self.sizes["u"])), dtype=torch.float64, device=device)
        self.out_l = torch.zeros(max(1, sum(self.sizes["m"])), dtype=torch.float64, device=device)
        self.x0 = pool([qp.x0 for qp in self.qps], device)
        self._graphs = []

    # -- helpers ---------------------------------------------------------
    def _split(self, t: torch.Tensor, key: str, shapes):
        out, o = [], 0
        host = t.cpu().numpy()
        for n, shp in zip(self.sizes[key], shapes):
            out.append(host[o:o + n].reshape(shp))
            o += n
        return out

    def set_x0(self, x0s):
        self.x0 = pool(list(x0s), self.device)

    # -- API ---------------------------------------------------------------
    def solve(self, iters: int = 0, tol: float = 0.0, fetch: bool = True) -> Result | int:
        info = (native.qp_info * self.B)()
        st = self.lib.qp_solve(self.h, _dptr(self.x0), int(iters), float(tol), _dptr(self.out_x),
                               _dptr(self.out_u), _dptr(self.out_l), info)
        native.check(st, "qp_solve")
        if not fetch:
            return st
        dx = self._split(self.out_x, "x", [(qp.N + 1, qp.nx) for qp in self.qps])
        du = self._split(self.out_u, "u", [(qp.N, qp.nu) for qp in self.qps])
        lam = self._split(self.out_l, "m", [(qp.m,) for qp in self.qps])
        infos = [dict(status=info[i].status, iters=info[i].iters, refactors=info[i].refactors,
                      refines=info[i].refines, fallback=info[i].fallback, rho=info[i].rho,
                      r_prim=info[i].r_prim, r_dual=info[i].r_dual, kkt=info[i].kkt) for i in range(self.B)]
        return Result(dx, du, lam, infos, st)

    def riccati(self):
        P = torch.zeros(max(1, sum(self.sizes["P"])), dtype=torch.float64, device=self.device)
        K = torch.zeros(max(1, sum(self.sizes["K"])), dtype=torch.float64, device=self.device)
        native.check(self.lib.qp_riccati(self.h, _dptr(P), _dptr(K)), "qp_riccati")
        Ps = self._split(P, "P", [(qp.N + 1, qp.nx, qp.nx) for qp in self.qps])
        Ks = self._split(K, "K", [(qp.N, qp.nu, qp.nx) for qp in self.qps])
        return Ps, Ks

    def kkt(self, dx, du, lam):
        out = (C.c_double * self.B)()
        tx = pool(list(dx), self.device)
        tu = pool(list(du), self.device)
        tl = pool(list(lam), self.device)
        native.check(self.lib.qp_kkt(self.h, _dptr(self.x0), _dptr(tx), _dptr(tu), _dptr(tl), out), "qp_kkt")
        return [out[i] for i in range(self.B)]

    def set_warm_start(self, z=None, y=None, rho=None):
        tz = pool(list(z), self.device) if z is not None else None
        ty = pool(list(y), self.device) if y is not None else None
        ra = None
        if rho is not None:
            vals = [float(rho)] * self.B if np.isscalar(rho) else [float(v) for v in rho]
            ra = (C.c_double * self.B)(*vals)
        native.check(self.lib.qp_set_warm_start(self.h, _dptr(tz), _dptr(ty), ra), "qp_set_warm_start")

    def get_state(self):
        tz = torch.zeros(max(1, sum(self.sizes["m"])), dtype=torch.float64, device=self.device)
        ty = torch.zeros_like(tz)
        rho = (C.c_double * self.B)()
        native.check(self.lib.qp_get_state(self.h, _dptr(tz), _dptr(ty), rho), "qp_get_state")
        return (self._split(tz, "m", [(qp.m,) for qp in self.qps]), self._split(ty, "m", [(qp.m,) for qp in self.qps]),
                [rho[i] for i in range(self.B)])

    def update(self, **arrays):
        """Replace problem arrays (keys A, B, c, Q, R, S, q, r, C, D, CN, lo, hi;
        each a list with one array per QP)."""
        keys = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi")
        unknown = set(arrays) - set(keys)
        if unknown:
            raise KeyError(sorted(unknown))
        t = {k: (pool(list(arrays[k]), self.device) if arrays.get(k) is not None else None) for k in keys}
        native.check(self.lib.qp_update(self.h, *[_dptr(t[k]) for k in keys]), "qp_update")

    def update_pools(self, pools: dict):
        """Same as update() with device pools already in the library's pool layout."""
        keys = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi")
        native.check(self.lib.qp_update(self.h, *[_dptr(pools.get(k)) for k in keys]), "qp_update")

    def reset(self):
        native.check(self.lib.qp_reset(self.h), "qp_reset")

    def features(self, idx=None) -> torch.Tensor:
        """qp_features of the QPs idx (default all) at the handle's x0:
        float32 device tensor [count, max nx + 4 P + 1] (rows padded with 0)."""
        ids = list(range(self.B)) if idx is None else [int(i) for i in idx]
        ld = max(self.nx[i] for i in ids) + 4 * native.GPUSLS_FEATURE_P + 1
        out = torch.zeros(len(ids), ld, dtype=torch.float32, device=self.device)
        tidx = torch.tensor(ids, dtype=torch.int32, device=self.device)
        native.check(self.lib.qp_features(self.h, _dptr(self.x0), _dptr(tidx), len(ids), ld, _dptr(out)),
                     "qp_features")
        return out

    def _heads_args(self, heads):
        """heads: list of (MLP, QP indices, n_stage) -> ctypes arrays (the
        index tensors are kept alive on the handle)."""
        n = len(heads)
        hs = (C.c_void_p * n)(*[hh[0].h.value for hh in heads])
        idx_t = [torch.tensor([int(i) for i in hh[1]], dtype=torch.int32, device=self.device) for hh in heads]
        self._keep = getattr(self, "_keep", []) + idx_t
        ids = (C.c_void_p * n)(*[t.data_ptr() for t in idx_t])
        counts = (C.c_int32 * n)(*[len(hh[1]) for hh in heads])
        ns = (C.c_int32 * n)(*[int(hh[2]) for hh in heads])
        return n, hs, ids, counts, ns

    def warm_start_heads(self, heads, rho_min=1e-3, rho_max=1e3):
        """qp_warm_start_heads: one network per shape family (list of
        (MLP, QP indices, n_stage)), features computed by the library."""
        n, hs, ids, counts, ns = self._heads_args(heads)
        native.check(self.lib.qp_warm_start_heads(self.h, n, hs, ids, counts, ns, _dptr(self.x0), float(rho_min),
                                                  float(rho_max)), "qp_warm_start_heads")

    def graph(self, mlp: "MLP | None" = None, features: torch.Tensor | None = None, rho_min=1e-3,
              rho_max=1e3, heads=None) -> "ServeGraph":
        """Capture one serving step (reset, optional learned warm start, solve)
        as a CUDA graph (qp_graph_create).  x0, the outputs and `features` are
        baked in: refill them in place (e.g. self.x0.copy_(...))."""
        g = ServeGraph(self, mlp, features, rho_min, rho_max, heads=heads)
        self._graphs.append(g)
        return g

    def close(self):
        for g in getattr(self, "_graphs", []):
            g.close()
        if getattr(self, "h", None) is not None:
            self.lib.qp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ServeGraph:
    """A QPBatch serving step captured as a CUDA graph: launch() replays reset,
    the learned warm start (when an MLP was given) and the persistent solve on
    a stream, with no host synchronization; info() reads the per-QP results."""

    def __init__(self, qb: QPBatch, mlp=None, features=None, rho_min=1e-3, rho_max=1e3, heads=None):
        self.lib = qb.lib
        self.qb = qb
        self.features = features
        self.info_i = torch.zeros(qb.B * 8, dtype=torch.int32, device=qb.device)
        self.info_d = torch.zeros(qb.B * 4, dtype=torch.float64, device=qb.device)
        g = C.c_void_p()
        if heads:
            n, hs, ids, counts, ns = qb._heads_args(heads)
            st = self.lib.qp_graph_create_heads(C.byref(g), qb.h, n, hs, ids, counts, ns, _dptr(qb.x0),
                                                _dptr(qb.out_x), _dptr(qb.out_u), _dptr(qb.out_l),
                                                _dptr(self.info_i), _dptr(self.info_d), float(rho_min),
                                                float(rho_max))
            native.check(st, "qp_graph_create_heads")
        else:
            st = self.lib.qp_graph_create(C.byref(g), qb.h, mlp.h if mlp is not None else None, _dptr(features),
                                          _dptr(qb.x0), _dptr(qb.out_x), _dptr(qb.out_u), _dptr(qb.out_l),
                                          _dptr(self.info_i), _dptr(self.info_d), float(rho_min), float(rho_max))
            native.check(st, "qp_graph_create")
        self.g = g

    def launch(self, stream: torch.cuda.Stream | None = None):
        native.check(self.lib.qp_graph_launch(self.g, _stream_ptr(stream or self.qb.stream)), "qp_graph_launch")

    def kernel_count(self) -> int:
        """Kernel launches per replay, counted from the captured graph."""
        n = C.c_int32()
        native.check(self.lib.qp_graph_kernel_count(self.g, C.byref(n)), "qp_graph_kernel_count")
        return int(n.value)

    def info(self) -> list[dict]:
        ii = self.info_i.view(self.qb.B, 8).cpu().numpy()
        dd = self.info_d.view(self.qb.B, 4).cpu().numpy()
        return [dict(status=int(a[0]), iters=int(a[1]), refactors=int(a[2]), refines=int(a[3]), fallback=int(a[4]),
                     rho=float(b[0]), r_prim=float(b[1]), r_dual=float(b[2]), kkt=float(b[3])) for a, b in zip(ii, dd)]

    def close(self):
        if getattr(self, "g", None) is not None:
            self.lib.qp_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SLS:
    """SLS controller synthesis and reachability margins (sls_setup / sls_solve)."""

    def __init__(self, nx, nu, N, nc, nf, per_j_tau: bool, precision=native.GPUSLS_FP64, stream=None,
                 device="cuda", inner: native.qp_settings | None = None):
        self.lib = native.load()
        self.dims = (nx, nu, N, nc, nf)
        self.device = device
        d = native.qp_dims(nx, nu, N, nc, nf)
        h = C.c_void_p()
        native.check(self.lib.sls_setup_ex(C.byref(h), d, int(precision), int(bool(per_j_tau)),
                                           C.byref(inner) if inner is not None else None, _stream_ptr(stream)),
                     "sls_setup_ex")
        self.h = h

    def solve(self, sp, fetch=True):
        """sp: an SLSProblem whose arrays are numpy arrays or device tensors
        (float64, in the sls_solve layouts; device tensors are used in place)."""
        nx, nu, N, nc, nf = self.dims

        def f(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return a
            return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.device)

        t = dict(A=f(sp.A), B=f(sp.B), E=f(sp.E), Qbar=f(sp.Qbar), Rbar=f(sp.Rbar), QbarN=f(sp.QbarN),
                 C=f(sp.C), D=f(sp.D), CN=f(sp.CN), tau=f(sp.tau))
        Phix = torch.empty(N * nx, N * nx, dtype=torch.float64, device=self.device)
        Phiu = torch.empty(N * nu, N * nx, dtype=torch.float64, device=self.device)
        h = torch.empty(max(1, N * nc), dtype=torch.float64, device=self.device)
        hf = torch.empty(max(1, nf), dtype=torch.float64, device=self.device)
        native.check(self.lib.sls_solve(self.h, *[_dptr(t[k]) for k in ("A", "B", "E", "Qbar", "Rbar", "QbarN", "C",
                                                                          "D", "CN", "tau")],
                                        _dptr(Phix), _dptr(Phiu), _dptr(h), _dptr(hf)), "sls_solve")
        if not fetch:
            return None
        return (Phix.cpu().numpy(), Phiu.cpu().numpy(), h.cpu().numpy()[:N * nc].reshape(N, nc),
                hf.cpu().numpy()[:nf])

    def tau(self, lam, eps: float = 1e-8) -> np.ndarray:
        """sls_tau: App. B duals from the last solve and multipliers lam."""
        nx, nu, N, nc, nf = self.dims
        w = max(nc, nf, 1)
        tl = _dev64(lam, self.device)
        out = torch.empty((N + 1) * N * w, dtype=torch.float64, device=self.device)
        native.check(self.lib.sls_tau(self.h, _dptr(tl), float(eps), _dptr(out)), "sls_tau")
        return out.cpu().numpy().reshape(N + 1, N, w)

    def close(self):
        if getattr(self, "h", None) is not None:
            self.lib.sls_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dev64(a, device):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return a
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)


class FastSLS:
    """The FastSLS alternation (fastsls_solve): one nominal QP handle and one
    per-j-tau SLS handle over the same dynamics and constraints.  step()
    runs `iters` alternation steps and returns the last step's outputs; the
    duals it returns are the next call's tau_in (the RTI chaining)."""

    def __init__(self, qp, sp, settings: native.qp_settings | None = None, sls_precision=native.GPUSLS_FP64,
                 stream=None, device="cuda", eps_tau: float = 1e-8):
        self.lib = native.load()
        self.device = device
        self.qb = QPBatch([qp], settings, stream=stream, device=device)
        self.sls = SLS(qp.nx, qp.nu, qp.N, qp.nc, qp.nf, per_j_tau=True, precision=sls_precision, stream=stream,
                       device=device)
        self.eps_tau = float(eps_tau)
        self.dims = qp.dims()
        nx, nu, N, nc, nf = self.dims
        self.w = max(nc, nf, 1)
        self.data = {k: _dev64(getattr(sp, k), device) for k in ("A", "B", "E", "Qbar", "Rbar", "QbarN", "C", "D",
                                                                 "CN")}
        self.lo = _dev64(qp.lo, device)
        self.hi = _dev64(qp.hi, device)
        self.x0 = _dev64(qp.x0, device)
        self.tau = torch.zeros((N + 1) * N * self.w, dtype=torch.float64, device=device)
        self.Phix = torch.empty(N * nx, N * nx, dtype=torch.float64, device=device)
        self.Phiu = torch.empty(N * nu, N * nx, dtype=torch.float64, device=device)
        self.hk = torch.zeros(max(1, N * nc), dtype=torch.float64, device=device)
        self.hf = torch.zeros(max(1, nf), dtype=torch.float64, device=device)

    def step(self, iters: int = 1, tau_in: torch.Tensor | None = None, fetch: bool = True, phi: bool = True):
        info = (native.qp_info * 1)()
        d = self.data
        qb = self.qb
        st = self.lib.fastsls_solve(qb.h, self.sls.h, *[_dptr(d[k]) for k in ("A", "B", "E", "Qbar", "Rbar", "QbarN",
                                                                                "C", "D", "CN")],
                                    _dptr(self.lo), _dptr(self.hi), _dptr(self.x0), int(iters), self.eps_tau,
                                    _dptr(tau_in), _dptr(self.tau), _dptr(qb.out_x), _dptr(qb.out_u),
                                    _dptr(qb.out_l), _dptr(self.Phix) if phi else None,
                                    _dptr(self.Phiu) if phi else None, _dptr(self.hk),
                                    _dptr(self.hf) if self.dims[4] else None, info)
        native.check(st, "fastsls_solve")
        if not fetch:
            return st
        nx, nu, N, nc, nf = self.dims
        return dict(x=qb.out_x.cpu().numpy()[:(N + 1) * nx].reshape(N + 1, nx),
                    u=qb.out_u.cpu().numpy()[:N * nu].reshape(N, nu), lam=qb.out_l.cpu().numpy()[:N * nc + nf],
                    tau=self.tau.cpu().numpy().reshape(N + 1, N, self.w),
                    Phix=self.Phix.cpu().numpy() if phi else None, Phiu=self.Phiu.cpu().numpy() if phi else None,
                    h=self.hk.cpu().numpy()[:N * nc].reshape(N, nc), hf=self.hf.cpu().numpy()[:nf],
                    info=dict(status=info[0].status, iters=info[0].iters, refactors=info[0].refactors,
                              kkt=info[0].kkt), status=st)

    def close(self):
        self.qb.close()
        self.sls.close()


def model_spec(ms) -> native.model_spec:
    """The C struct of a workloads.ModelSpec (field by field)."""
    m = native.model_spec()
    m.kind = native.GPUSLS_MODEL_DUBINS if ms.kind == "dubins" else native.GPUSLS_MODEL_QUAD2D
    m.N, m.n_obs = int(ms.N), int(ms.n_obs)
    if m.n_obs > native.GPUSLS_MODEL_MAX_OBS:
        raise ValueError("too many obstacles")
    m.dt, m.v, m.mass, m.grav, m.arm, m.inertia = (float(ms.dt), float(ms.v), float(ms.mass), float(ms.grav),
                                                   float(ms.arm), float(ms.inertia))
    for name in ("u_lo", "u_hi", "xref", "uref", "Qd", "Rd", "QNd"):
        arr = getattr(m, name)
        for i, v in enumerate(np.asarray(getattr(ms, name), dtype=float).ravel()):
            arr[i] = float(v)
    for i, v in enumerate(np.asarray(ms.E, dtype=float).ravel()):
        m.E[i] = float(v)
    for i, v in enumerate(np.asarray(ms.obstacles, dtype=float).ravel()):
        m.obs[i] = float(v)
    return m


def linearize(ms, X, U, x0bar, device="cuda"):
    """model_linearize on a batch of nominal trajectories (numpy [batch, ...]);
    returns one dict of numpy arrays per trajectory (the LTV-QP arrays and
    the initial deviation dx0)."""
    lib = native.load()
    m = model_spec(ms)
    d = native.qp_dims()
    native.check(lib.model_dims(C.byref(m), C.byref(d)), "model_dims")
    X = np.asarray(X, dtype=np.float64)
    Bn = X.shape[0]
    nx, nu, N, nc, nf = d.nx, d.nu, d.N, d.nc, d.nf
    shapes = dict(A=(N, nx, nx), B=(N, nx, nu), c=(N, nx), Q=(N + 1, nx, nx), R=(N, nu, nu), S=(N, nu, nx),
                  q=(N + 1, nx), r=(N, nu), C=(N, nc, nx), D=(N, nc, nu), CN=(nf, nx), lo=(N * nc + nf,),
                  hi=(N * nc + nf,), dx0=(nx,))
    out = {k: torch.empty(max(1, Bn * int(np.prod(v))), dtype=torch.float64, device=device)
           for k, v in shapes.items()}
    tX, tU, tx = _dev64(X, device), _dev64(U, device), _dev64(x0bar, device)
    keys = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi", "dx0")
    native.check(lib.model_linearize(C.byref(m), Bn, _dptr(tX), _dptr(tU), _dptr(tx), *[_dptr(out[k]) for k in keys],
                                     _stream_ptr(None)), "model_linearize")
    res = []
    for b in range(Bn):
        res.append({k: out[k].cpu().numpy()[b * int(np.prod(v)):(b + 1) * int(np.prod(v))].reshape(v)
                    for k, v in shapes.items()})
    return res


class SQP:
    """sqp_setup / sqp_solve / rti_step over a batch of trajectories of one
    model (workloads.ModelSpec).  X [batch, N+1, nx], U [batch, N, nu] and
    the states x [batch, nx] live on the device (torch tensors) and are
    updated in place by the library."""

    def __init__(self, ms, batch: int, settings: native.qp_settings | None = None, robust: bool = False,
                 stream=None, device="cuda"):
        self.lib = native.load()
        self.ms = ms
        self.spec = model_spec(ms)
        self.batch = batch
        self.device = device
        self.settings = settings or native.default_settings()
        d = native.qp_dims()
        native.check(self.lib.model_dims(C.byref(self.spec), C.byref(d)), "model_dims")
        self.dims = (d.nx, d.nu, d.N, d.nc, d.nf)
        h = C.c_void_p()
        native.check(self.lib.sqp_setup(C.byref(h), C.byref(self.spec), batch, C.byref(self.settings), int(robust),
                                        _stream_ptr(stream)), "sqp_setup")
        self.h = h
        nx, nu, N, nc, nf = self.dims
        self.X = torch.zeros(batch, N + 1, nx, dtype=torch.float64, device=device)
        self.U = torch.zeros(batch, N, nu, dtype=torch.float64, device=device)
        self.x = torch.zeros(batch, nx, dtype=torch.float64, device=device)
        self.u0 = torch.zeros(batch, nu, dtype=torch.float64, device=device)
        self.hk = torch.zeros(max(1, N * nc), dtype=torch.float64, device=device)
        self.hf = torch.zeros(max(1, nf), dtype=torch.float64, device=device)

    def set_nominal(self, X, U):
        self.X.copy_(torch.as_tensor(np.asarray(X, dtype=np.float64).reshape(self.X.shape)))
        self.U.copy_(torch.as_tensor(np.asarray(U, dtype=np.float64).reshape(self.U.shape)))

    def set_state(self, x):
        self.x.copy_(torch.as_tensor(np.asarray(x, dtype=np.float64).reshape(self.x.shape)))

    def solve(self, iters: int, merit_w: float = 100.0, line_search: bool = True):
        """sqp_solve from the current nominal and states; returns the step
        sizes [iters, batch] and the last QP infos."""
        a = (C.c_double * (iters * self.batch))()
        info = (native.qp_info * self.batch)()
        st = self.lib.sqp_solve(self.h, _dptr(self.X), _dptr(self.U), _dptr(self.x), int(iters), float(merit_w),
                                int(bool(line_search)), a, info)
        native.check(st, "sqp_solve")
        return np.array(a[:]).reshape(iters, self.batch), [dict(status=i.status, iters=i.iters, kkt=i.kkt)
                                                            for i in info]

    def rti_step(self, W=None):
        """rti_step with the disturbances W [batch, nx] (numpy or device
        tensor; None: no disturbance); returns the QP infos."""
        tW = None if W is None else _dev64(np.asarray(W, dtype=np.float64) if not isinstance(W, torch.Tensor) else W,
                                           self.device)
        info = (native.qp_info * self.batch)()
        st = self.lib.rti_step(self.h, _dptr(self.X), _dptr(self.U), _dptr(self.x), _dptr(tW), _dptr(self.u0),
                               _dptr(self.hk), _dptr(self.hf), info)
        native.check(st, "rti_step")
        return [dict(status=i.status, iters=i.iters, kkt=i.kkt) for i in info]

    def reset_duals(self):
        native.check(self.lib.sqp_reset_duals(self.h), "sqp_reset_duals")

    def close(self):
        if getattr(self, "h", None) is not None:
            self.lib.sqp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The warm-start network (mlp_* in include/gpusls.h); FP32 device tensors."""

    def __init__(self, n_in, hidden, n_out, max_batch, stream=None, device="cuda"):
        self.lib = native.load()
        self.n_in, self.hidden, self.n_out, self.max_batch = n_in, hidden, n_out, max_batch
        self.device = device
        self.stream = stream
        h = C.c_void_p()
        native.check(self.lib.mlp_create(C.byref(h), n_in, hidden, n_out, max_batch, _stream_ptr(stream)),
                     "mlp_create")
        self.h = h

    def shapes(self):
        i, hdn, o = self.n_in, self.hidden, self.n_out
        return [(hdn, i), (hdn,), (hdn, hdn), (hdn,), (o, hdn), (o,)]

    def set_params(self, params):
        ts = [torch.as_tensor(np.ascontiguousarray(p, dtype=np.float32)).to(self.device) for p in params]
        native.check(self.lib.mlp_set_params(self.h, *[_dptr(t) for t in ts]), "mlp_set_params")

    def get_params(self):
        ts = [torch.empty(shp, dtype=torch.float32, device=self.device) for shp in self.shapes()]
        native.check(self.lib.mlp_get_params(self.h, *[_dptr(t) for t in ts]), "mlp_get_params")
        return [t.cpu().numpy() for t in ts]

    def fit_normalization(self, X: torch.Tensor, T: torch.Tensor):
        native.check(self.lib.mlp_fit_normalization(self.h, _dptr(X), _dptr(T), X.shape[0]), "mlp_fit_normalization")

    def set_normalization(self, xm, xs, ym, ys):
        ts = [torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(self.device) for a in (xm, xs, ym, ys)]
        native.check(self.lib.mlp_set_normalization(self.h, *[_dptr(t) for t in ts]), "mlp_set_normalization")

    def save(self, path: str):
        """The network (parameters and normalization) to a binary file (mlp_save)."""
        native.check(self.lib.mlp_save(self.h, os.fsencode(path)), "mlp_save")

    def load(self, path: str):
        """Parameters and normalization from a file written by save (mlp_load)."""
        native.check(self.lib.mlp_load(self.h, os.fsencode(path)), "mlp_load")

    def get_normalization(self):
        ts = [torch.empty(n, dtype=torch.float32, device=self.device)
              for n in (self.n_in, self.n_in, self.n_out, self.n_out)]
        native.check(self.lib.mlp_get_normalization(self.h, *[_dptr(t) for t in ts]), "mlp_get_normalization")
        return [t.cpu().numpy() for t in ts]

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        Y = torch.empty(X.shape[0], self.n_out, dtype=torch.float32, device=self.device)
        native.check(self.lib.mlp_forward(self.h, _dptr(X), X.shape[0], _dptr(Y)), "mlp_forward")
        return Y

    def gradients(self, Xn: torch.Tensor, Tn: torch.Tensor):
        n = sum(int(np.prod(s)) for s in self.shapes())
        g = torch.empty(n, dtype=torch.float32, device=self.device)
        loss = C.c_float()
        native.check(self.lib.mlp_gradients(self.h, _dptr(Xn), _dptr(Tn), Xn.shape[0], _dptr(g), C.byref(loss)),
                     "mlp_gradients")
        out, o, host = [], 0, g.cpu().numpy()
        for shp in self.shapes():
            k = int(np.prod(shp))
            out.append(host[o:o + k].reshape(shp))
            o += k
        return out, loss.value

    def train_step(self, X: torch.Tensor, T: torch.Tensor, lr: float) -> float:
        loss = C.c_float()
        native.check(self.lib.mlp_train_step(self.h, _dptr(X), _dptr(T), X.shape[0], float(lr), C.byref(loss)),
                     "mlp_train_step")
        return loss.value

    def warm_start(self, qb: "QPBatch", features: torch.Tensor, rho_min=1e-3, rho_max=1e3):
        native.check(self.lib.qp_warm_start_mlp(qb.h, self.h, _dptr(features), rho_min, rho_max),
                     "qp_warm_start_mlp")

    def close(self):
        if getattr(self, "h", None) is not None:
            self.lib.mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
