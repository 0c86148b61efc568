#!/usr/bin/env python
"""Benchmark: ms per QP solved to a 1e-4 FP64 KKT residual on quadruped-shaped
(nx=61, nu=12, N=100) LTV-QPs -- the learned-warm-start, batched, FP32 GPU
solver (headline) next to the same batch solved cold, the plain FP64
single-QP GPU solve, and the FP64 CPU oracle.

One step = warm-start inference (MLP) + one solve (factorization + ADMM
iterations + FP64 KKT gate with refinement) of every QP in the batch, from a
reset state.  Problem data for the whole batch stays resident
on the device (2.2 GB in FP64 for 256 QPs, larger than L2); `e2e` repeats the step through
the public API with the problem data copied from pinned host memory and the
solution copied back inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpusls|reference]
"""
from __future__ import annotations

import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ms/QP solve to 1e-4 KKT residual (61D, N=100): learned+batched vs plain ADMM"
EPS_KKT = 1e-4           # the certified FP64 KKT tolerance of the metric
# In-loop residual tolerance of every 1e-4 solve here (GPU, plain FP64 GPU
# and the CPU oracle alike): half the KKT tolerance.  At eps = 1e-4 the first
# KKT gate usually fails and the tightening overshoots to 1e-5; chosen on
# validation instances 300000..300255 (1e-4: 0.477, 5e-5: 0.455, 3e-5: 0.451,
# 2e-5: 0.459 ms/QP) and the learned serving mix (0.556, 0.545, 0.552).
EPS_IN = 0.5 * EPS_KKT
# Stop-test interval of the same solves (every solve's residual check, KKT
# gate and stop decision; OSQP checks every 25): 10 instead of the library's
# default 5, chosen on the same validation instances (5: 0.453, 10: 0.441,
# 15: 0.438 ms/QP at the same iteration counts).
CHECK_EVERY = 10
# rho-update interval (every sigma iterations) of the same solves: 50 instead
# of the library's default 25, chosen on the same validation instances
# (learned 25: 0.443, 50: 0.428, 100: 0.421 ms/QP at the same iterations;
# cold 25: 0.818 / 381 iterations, 50: 0.735 / 342, 100: 0.804 / 408).
SIGMA = 50
WORKLOAD = "quadruped-shaped LTV-QP family (nx=61 nu=12 N=100 nc=20 nf=8), held-out instances 100000 + i"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6400.0
TRAFFIC_PER_QP_ITER = 6.03e6   # bytes, ncu DRAM read+write per QP-iteration (61D, N=100, FP32, cluster 6, 45 QPs)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpusls", choices=["gpusls", "reference"])
    p.add_argument("--batch", type=int, default=256)
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed"])
    p.add_argument("--cluster", type=int, default=8)
    p.add_argument("--plain-qps", type=int, default=2)
    p.add_argument("--cpu-sample", type=int, default=32)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--fallback", type=int, default=2000)
    p.add_argument("--no-autotune", action="store_true", help="keep --cluster instead of tuning the launch shape")
    p.add_argument("--eager", action="store_true", help="time the step as separate calls instead of the graph")
    p.add_argument("--no-extras", action="store_true", help="skip the serving-mix / humanoid / SLS measurements")
    p.add_argument("--index-order", action="store_true",
                   help="launch QPs in index order instead of longest-expected-first")
    p.add_argument("--case", default="", choices=["", "iter", "refactor", "mlp", "sls", "long"],
                   help="small fixed case for profiler captures (prints no bench line)")
    p.add_argument("--case-batch", type=int, default=32, help="QPs of the iter / refactor profiling cases")
    p.add_argument("--model", default=os.path.join(ROOT, "paper_2604_07644_b300", "warmstart_quadruped61.npz"))
    return p.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[2 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def algorithmic_bytes_per_iter(nx, nu, N, nc, esz):
    """Operators one cached ADMM iteration must read once per QP (FP32 storage):
    N (2 nx^2 + 3 nu nx + nu nc + 2 nc (nx + nu)) elements."""
    return N * (2 * nx * nx + 3 * nu * nx + nu * nc + 2 * nc * (nx + nu)) * esz


def _oracle_worker_init():
    """Pool worker start-up: the oracle's imports, outside the timed region."""
    sys.path.insert(0, ROOT)
    import oracle.admm  # noqa: F401
    from paper_2604_07644_b300 import workloads  # noqa: F401


def _oracle_worker(idx):
    """One family instance solved by the FP64 oracle ADMM to the 1e-4 KKT
    tolerance (the instance is regenerated here from its index)."""
    from oracle import admm
    from paper_2604_07644_b300 import workloads as W
    qp = W.family(0).instance(idx)
    r = admm.admm(qp, admm.Settings(eps=EPS_IN, eps_kkt=EPS_KKT, check_every=CHECK_EVERY, sigma=SIGMA))
    return idx, r.iters, r.x, r.u


def cpu_oracle_pool(indices):
    """The FP64 oracle as it stands over the host's cores: one QP per worker
    process (spawned, so it is safe after CUDA initialisation), as many
    workers as cores or QPs.  Returns (ms per QP of wall time, workers,
    results [(index, iters, x, u)])."""
    import multiprocessing as mp
    procs = max(1, min(len(os.sched_getaffinity(0)), len(indices)))
    with mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init) as pool:
        pool.map(abs, range(procs))                      # workers up before the clock starts
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, indices, chunksize=1)
        dt = time.perf_counter() - t0
    return dt * 1e3 / len(indices), procs, res


def host_cpu():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "usable": len(os.sched_getaffinity(0)), "model": model}


def cpu_oracle_ms_per_qp(qps, eps=EPS_KKT, results=None):
    """The FP64 oracle as it stands on this host (single thread); the solutions
    are appended to `results` when given."""
    from oracle import admm
    t0 = time.perf_counter()
    iters = []
    for qp in qps:
        r = admm.admm(qp, admm.Settings(eps=0.5 * eps, eps_kkt=eps, check_every=CHECK_EVERY, sigma=SIGMA))
        iters.append(r.iters)
        if results is not None:
            results.append(r)
    dt = time.perf_counter() - t0
    return dt * 1e3 / len(qps), iters


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle on the same workload, one QP per step."""
    if rank != 0:
        return
    from paper_2604_07644_b300 import workloads as W
    fam = W.family(0)
    # the QPs of this arm's batch (held-out instances 100000 + i), one per
    # step; warm-up steps solve instances that the timed steps do not
    for w in range(args.warmup):
        cpu_oracle_ms_per_qp([fam.instance(100000 + args.batch - 1 - w)])
    t0 = time.perf_counter()
    iters = []
    for n in range(args.steps):
        _, it = cpu_oracle_ms_per_qp([fam.instance(100000 + n)])
        iters += it
    dt = time.perf_counter() - t0
    ms = dt * 1e3 / args.steps
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms/QP", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": args.batch, "precision": "fp64",
                       "solver": "CPU oracle ADMM (sequential Riccati), the same solver settings"},
            "cpu_baseline": {"value": ms, "unit": "ms/QP", "cores": 1, "kind": "oracle",
                             "sample": f"the first {args.steps} QPs of the batch, one per step, single thread; "
                                       f"iters {iters}"},
            "e2e": {"value": ms, "unit": "ms/QP", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time_graph(g, stream, steps):
    import torch
    g.launch(stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def split_solution(sol, qps):
    """Per-QP (X [N+1][nx], U [N][nu]) from a batch's stacked dx, du."""
    x, u = sol
    ox, ou = 0, 0
    xs, us = [], []
    for qp in qps:
        xs.append(x[ox:ox + (qp.N + 1) * qp.nx].reshape(qp.N + 1, qp.nx))
        us.append(u[ou:ou + qp.N * qp.nu].reshape(qp.N, qp.nu))
        ox += (qp.N + 1) * qp.nx
        ou += qp.N * qp.nu
    return xs, us


def exact_distance(xs, us, n_qps):
    """Largest distance, relative to max(1, max|x*|), of the sampled QPs'
    solutions from the exact optima stored in tests/golden/exact_quadruped61.npz
    (instances 100000 + i); (None, []) without the file."""
    gold_path = os.path.join(ROOT, "tests", "golden", "exact_quadruped61.npz")
    if not os.path.exists(gold_path):
        return None, []
    gold = np.load(gold_path)
    d, ids = 0.0, []
    for j, i in enumerate(gold["ids"]):
        i = int(i)
        if i >= n_qps:
            continue
        ids.append(i)
        scale = max(1.0, float(np.max(np.abs(gold["x"][j]))))
        d = max(d, float(np.max(np.abs(xs[i] - gold["x"][j]))) / scale,
                float(np.max(np.abs(us[i] - gold["u"][j]))) / scale)
    return d, ids


def extra_workloads(args, qps, sol, stream, dev, oracle_sols):
    """Timed on the same device after the headline: the batched serving mix
    (256 ragged QPs, nx in {12, 61, 75}, N in 16..128, cold FP32), 64
    humanoid-shaped QPs (75D, N=40, cold FP32), the plain 4D QP (FP64, 200
    iterations) and 64 quadrotor-shaped QPs (12D, N=64; FP32 and FP64), the
    humanoid SLS solve (75D, N=40) with per-j tau and with tau = 0, and
    checks of the headline's
    solutions: the largest bound violation and the largest difference from
    the FP64 oracle on the CPU-baseline sample."""
    import torch

    from paper_2604_07644_b300 import native
    from paper_2604_07644_b300 import workloads as W
    from paper_2604_07644_b300.api import SLS, QPBatch
    out = {}
    steps = max(1, args.steps)
    base = dict(precision=native.GPUSLS_FP32, cluster=8, max_refine=3, max_iter=6000, schedule=1, eps=EPS_IN,
                eps_kkt=EPS_KKT, check_every=CHECK_EVERY, sigma=SIGMA)

    def batch_run(name, qps_, cluster, precision=native.GPUSLS_FP32):
        s = native.default_settings(**dict(base, cluster=cluster, precision=precision))
        if not args.no_autotune:
            from paper_2604_07644_b300 import autotune
            s, _ = autotune.choose(qps_, s, expected_iters=300, tail_iters=1500, cache=autotune.Cache())
        with torch.cuda.stream(stream):
            qb = QPBatch(qps_, s, stream=stream, device=dev)
            g = qb.graph()
            ms = _time_graph(g, stream, steps)
            info = g.info()
        out[name] = {"ms_per_qp": ms / len(qps_), "batch": len(qps_), "cluster": int(s.cluster),
                     "occupancy": int(s.occupancy),
                     "iters_mean": float(np.mean([i["iters"] for i in info])),
                     "kkt_max": float(np.max([i["kkt"] for i in info])),
                     "all_converged": all(i["status"] == 0 for i in info)}
        qb.close()

    batch_run("serving_mix_cold", W.serving_mix(0, 256), 8)

    # the learned serving mix: 256 QPs of three shape families (12D/4, 61D/12,
    # 75D/21) with N ~ U{16..128}, one warm-start head per family inside the
    # graph, against the same batch cold
    from paper_2604_07644_b300 import learned as L
    mixl = W.serving_mix_learned(0, 256)
    qpl_ = [q for q, _ in mixl]
    s = native.default_settings(**dict(base, cluster=4))
    if not args.no_autotune:
        from paper_2604_07644_b300 import autotune
        s, _ = autotune.choose(qpl_, s, expected_iters=200, tail_iters=1500, cache=autotune.Cache())
    with torch.cuda.stream(stream):
        qb = QPBatch(qpl_, s, stream=stream, device=dev)
        heads_ = L.mix_heads(mixl, os.path.join(ROOT, "paper_2604_07644_b300"), stream=stream)
        for name, g in (("serving_mix_learned", qb.graph(heads=heads_)), ("serving_mix_learned_cold", qb.graph())):
            ms = _time_graph(g, stream, steps)
            info = g.info()
            out[name] = {"ms_per_qp": ms / len(qpl_), "batch": len(qpl_), "cluster": int(s.cluster),
                         "occupancy": int(s.occupancy), "iters_mean": float(np.mean([i["iters"] for i in info])),
                         "kkt_max": float(np.max([i["kkt"] for i in info])),
                         "all_converged": all(i["status"] == 0 for i in info)}
        for h_ in heads_:
            h_[0].close()
        qb.close()

    # long horizon (the horizon study of Sec. V-A): torque-limited
    # pendulum-shaped QP, nx=30, nu=15, N=3000 (1.35e5 decision variables),
    # cold FP32 solve to the 1e-4 KKT tolerance, one QP per launch; the
    # automatic launch shape (cluster = 0) takes 16-CTA clusters here
    qpl = W.long_horizon(0)
    for tol, key in ((1e-4, "long_horizon_N3000"), (1e-2, "long_horizon_N3000_tol1e-2")):
        # 1e-2: the residual tolerance of the paper's horizon study (Sec. V-A)
        sl = native.default_settings(precision=native.GPUSLS_FP32, cluster=0, eps=tol, eps_kkt=tol,
                                     eps_floor=min(1e-5, 0.1 * tol), max_iter=20000)
        with torch.cuda.stream(stream):
            ql = QPBatch([qpl], sl, stream=stream, device=dev)
            gl = ql.graph()
            ms = _time_graph(gl, stream, steps)
            il = gl.info()[0]
        out[key] = {"ms_per_qp": ms, "iters": il["iters"], "kkt": il["kkt"], "status": il["status"],
                    "variables": (qpl.N + 1) * qpl.nx + qpl.N * qpl.nu, "kkt_tolerance": tol,
                    "cluster": "automatic (16 CTAs, non-portable cluster size)",
                    "workload": "pendulum-shaped LTV-QP nx=30 nu=15 N=3000, |u| <= 1, cold FP32"}
        ql.close()
    batch_run("humanoid75_cold", [W.humanoid_75d(s) for s in range(64)], 4)

    # the two small configurations: the plain 4D QP (FP64, 200 iterations,
    # one instance per launch) and 64 quadrotor-shaped QPs (12D, N=64) in
    # FP32 and in FP64, cold, to the 1e-4 KKT tolerance
    s4 = native.default_settings(precision=native.GPUSLS_FP64, fixed_iters=200)
    with torch.cuda.stream(stream):
        q4 = QPBatch([W.plain_4d(0)], s4, stream=stream, device=dev)
        g4 = q4.graph()
        ms = _time_graph(g4, stream, max(steps, 10))
        i4 = g4.info()[0]
    out["plain4d_fp64_200iter"] = {"ms_per_solve": ms, "iters": i4["iters"], "kkt": i4["kkt"],
                                   "workload": "nx=4 nu=2 N=32, FP64, 200 ADMM iterations, one QP per launch"}
    q4.close()
    q12 = [W.quadrotor_12d(s) for s in range(64)]
    batch_run("quadrotor12_b64", q12, 4)
    batch_run("quadrotor12_b64_fp64", q12, 4, precision=native.GPUSLS_FP64)

    # SLS: model flops from the per-j scans (2 (N - j) combines of ~16.7 nx^3
    # each) and the forward products (2 nx^2 (nx + nu) per block)
    for mode in ("uniform", "zero"):
        sp = W.sls_problem(0, tau_mode=mode)
        N, nx = sp.A.shape[0], sp.A.shape[1]
        nu, nc, nf = sp.B.shape[2], sp.C.shape[1], sp.CN.shape[0]
        t = {k: (None if getattr(sp, k) is None else
                 torch.from_numpy(np.ascontiguousarray(getattr(sp, k), dtype=np.float64)).to(dev))
             for k in ("A", "B", "E", "Qbar", "Rbar", "QbarN", "C", "D", "CN", "tau")}
        from types import SimpleNamespace
        spd = SimpleNamespace(**t)
        sls = SLS(nx, nu, N, nc, nf, per_j_tau=(mode == "uniform"), precision=native.GPUSLS_FP32, stream=stream)
        with torch.cuda.stream(stream):
            sls.solve(spd, fetch=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                sls.solve(spd, fetch=False)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        scans = (sum(2 * (N - j) for j in range(N)) if mode == "uniform" else 2 * N) * 16.7 * nx ** 3
        fwd = (N * (N + 1) / 2) * 2 * nx * nx * (nx + nu)
        out[f"sls75_tau_{mode}"] = {"ms_per_solve": ms, "model_gflop": (scans + fwd) / 1e9,
                                   "model_gflops_per_s": (scans + fwd) / (ms * 1e-3) / 1e9}
        sls.close()

    # one RTI step of the FastSLS alternation at the humanoid size (nx=75,
    # nu=21, N=40; Sec. III-D / IV-C): SLS solve from the previous step's
    # duals, tightening, warm-started tightened QP solve, new duals
    from paper_2604_07644_b300.api import FastSLS
    qp75, sp75 = W.fastsls_problem(0, 75, 21, 40, w_range=(0.001, 0.01), tag=4)
    f = FastSLS(qp75, sp75, native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, max_iter=6000),
                sls_precision=native.GPUSLS_FP32, stream=stream)
    with torch.cuda.stream(stream):
        f.step(1, fetch=False)
        tau_prev = f.tau.clone()
        for _ in range(2):
            f.step(1, tau_in=tau_prev, fetch=False)
            tau_prev.copy_(f.tau)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            f.step(1, tau_in=tau_prev, fetch=False)
            tau_prev.copy_(f.tau)
        e1.record(stream)
        torch.cuda.synchronize()
    r = f.step(1, tau_in=tau_prev)
    out["fastsls75_rti_step"] = {"ms_per_step": e0.elapsed_time(e1) / steps, "qp_iters_last": r["info"]["iters"],
                                 "qp_kkt_last": r["info"]["kkt"], "h_max": float(np.max(r["h"])),
                                 "step": "sls_solve (per-j tau) + tighten + warm tightened QP solve (FP32) + sls_tau"}
    f.close()

    # RTI control steps (Sec. IV-C) on the paper's analytic models: the planar
    # quadrotor (App. D, N=25) robust (linearization + SLS update from the
    # previous duals + tightened QP + duals) and classical, and a batch of
    # 256 disturbed Dubins-car closed loops (App. C, N=30) per classical step
    from paper_2604_07644_b300.api import SQP
    s_rti = native.default_settings(precision=native.GPUSLS_FP64, max_iter=20000)
    mq = W.quad2d(0, N=25)
    for robust in (True, False):
        sq = SQP(mq, 1, s_rti, robust=robust, stream=stream)
        X0, U0 = mq.initial_guess()
        sq.set_nominal(X0[None], U0[None])
        sq.set_state(mq.x0[None])
        sq.solve(6)
        Wd = torch.from_numpy(W.disturbances(3, steps + 2, 1, mq.nx)).to(dev)
        with torch.cuda.stream(stream):
            for t in range(2):
                sq.rti_step(Wd[t])
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for t in range(steps):
                info = sq.rti_step(Wd[2 + t])
            e1.record(stream)
            torch.cuda.synchronize()
        out["quad2d_rti_" + ("robust" if robust else "classical")] = {
            "ms_per_step": e0.elapsed_time(e1) / steps, "qp_iters_last": info[0]["iters"],
            "step": "linearize + " + ("SLS(tau_prev) + tighten + " if robust else "") + "QP (FP64) + simulate + shift"}
        sq.close()
    md = W.dubins(0)
    Bd = 256
    sq = SQP(md, Bd, s_rti, stream=stream)
    X0, U0 = md.initial_guess()
    sq.set_nominal(np.repeat(X0[None], Bd, 0), np.repeat(U0[None], Bd, 0))
    sq.set_state(np.repeat(md.x0[None], Bd, 0))
    sq.solve(6)
    Wd = torch.from_numpy(W.disturbances(4, steps + 1, Bd, md.nx)).to(dev)
    with torch.cuda.stream(stream):
        sq.rti_step(Wd[0])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(steps):
            sq.rti_step(Wd[1 + t])
        e1.record(stream)
        torch.cuda.synchronize()
    out["dubins_rti_batch256"] = {"ms_per_step": e0.elapsed_time(e1) / steps, "rollouts": Bd,
                                  "ms_per_rollout_step": e0.elapsed_time(e1) / steps / Bd}
    sq.close()

    # checks on the headline's solutions (snapshot of the learned step's outputs)
    xs, us = split_solution(sol, qps)
    viol = 0.0
    for qp, X, U in zip(qps, xs, us):
        v = np.concatenate([np.einsum("kcx,kx->kc", qp.C, X[:-1]).ravel() + np.einsum("kcu,ku->kc", qp.D, U).ravel(),
                            qp.CN @ X[-1]])
        viol = max(viol, float(np.max(np.maximum(np.maximum(v - qp.hi, qp.lo - v), 0.0))))
    out["bound_violation_max"] = viol
    # distance to the exact optimum of eq. sqp_qp that the FP64 oracle stored
    # for sampled instances of this batch (tests/golden/exact_quadruped61.npz),
    # next to the oracle's own ADMM solves at the same 1e-4 KKT tolerance
    d_gpu, ids = exact_distance(xs, us, len(qps))
    if d_gpu is not None:
        gold = np.load(os.path.join(ROOT, "tests", "golden", "exact_quadruped61.npz"))
        base = 100000
        d_or, n_or = 0.0, 0
        by_idx = {r[0]: r for r in (oracle_sols or [])}
        for j, i in enumerate(gold["ids"]):
            r = by_idx.get(base + int(i))
            if int(i) >= len(qps) or r is None:
                continue
            n_or += 1
            scale = max(1.0, float(np.max(np.abs(gold["x"][j]))))
            d_or = max(d_or, float(np.max(np.abs(r[2] - gold["x"][j]))) / scale,
                       float(np.max(np.abs(r[3] - gold["u"][j]))) / scale)
        out["max_rel_diff_vs_exact"] = {
            "value": d_gpu, "qps": ids,
            "oracle_admm_same_tolerance": d_or if n_or else None, "oracle_qps": n_or,
            "note": "relative to max(1, max|x*|); x* = the exact optimum (oracle ADMM to 1e-11 + dense-KKT "
                    "active-set solve); a 1e-4 KKT residual bounds the distance only through the curvature"}
    return out


def profile_case(args):
    """Small fixed workloads for ncu captures (inputs larger than L2, a few
    hundred MB on the device):
      iter      32 (--case-batch) quadruped-shaped QPs (FP32, cluster 6), factorized by a first launch;
                launches 2 and 3 run 100 cached ADMM iterations each (no
                refactor), so a capture of launch 2 is the iteration alone;
      refactor  the same batch, three launches that each refactor and run one
                iteration;
      mlp       the learned warm start of 256 QPs (BF16 tensor-core GEMMs);
      sls       SLS synthesis at nx=75, nu=21, N=40 with per-j tau;
      long      the N=3000 pendulum-shaped QP (nx=30, nu=15), cold FP32 to
                the 1e-2 tolerance, automatic launch shape (16-CTA cluster),
                two solves."""
    import torch

    from paper_2604_07644_b300 import build as B_
    from paper_2604_07644_b300 import learned, native
    from paper_2604_07644_b300 import workloads as W
    from paper_2604_07644_b300.api import SLS, QPBatch
    B_.build()
    native.load()
    fam = W.family(0)
    if args.case in ("iter", "refactor"):
        qps = [fam.instance(100000 + i) for i in range(args.case_batch)]
        # the launch shape the autotuner picks for the bench's batch (cluster 6);
        # --case-batch 45 is the most 6-CTA clusters the device holds at once
        # (two CTAs on most SMs): one wave at the bench's occupancy
        prec = {"fp32": native.GPUSLS_FP32, "fp64": native.GPUSLS_FP64, "mixed": native.GPUSLS_MIXED}[args.precision]
        s = native.default_settings(precision=prec, cluster=6, sigma=0, fixed_iters=1)
        if args.case == "iter":
            s.fixed_iters = 100
        qb = QPBatch(qps, s)
        qb.reset()
        qb.solve(fetch=False)                         # launch 1: factorization + iterations
        for _ in range(2):                            # launches 2, 3
            if args.case == "refactor":
                qb.reset()                            # refactor again
            qb.solve(fetch=False)                     # iter: cached factorization, 100 iterations
        torch.cuda.synchronize()
        qb.close()
    elif args.case == "mlp":
        qps = [fam.instance(100000 + i) for i in range(256)]
        qb = QPBatch(qps, native.default_settings(precision=native.GPUSLS_FP32))
        qb.set_x0([q.x0 for q in qps])
        mlp = learned.load(args.model, max_batch=256)
        heads = [(mlp, list(range(len(qps))), qps[0].N)]
        for _ in range(3):
            qb.warm_start_heads(heads)
        torch.cuda.synchronize()
        mlp.close()
        qb.close()
    elif args.case == "long":
        qp = W.long_horizon(0)
        s = native.default_settings(precision=native.GPUSLS_FP32, cluster=0, eps=1e-2, eps_kkt=1e-2,
                                    eps_floor=1e-5, max_iter=20000)
        qb = QPBatch([qp], s)
        for _ in range(2):
            qb.reset()
            qb.solve(fetch=False)
        torch.cuda.synchronize()
        qb.close()
    elif args.case == "sls":
        p = W.sls_problem(0, tau_mode="uniform")
        N, nx = p.A.shape[0], p.A.shape[1]
        nu, nc, nf = p.B.shape[2], p.C.shape[1], p.CN.shape[0]
        sls = SLS(nx, nu, N, nc, nf, per_j_tau=True, precision=native.GPUSLS_FP32)
        for _ in range(2):
            sls.solve(p, fetch=False)
        torch.cuda.synchronize()
        sls.close()
    print(f"case {args.case} done", flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.case:
        profile_case(args)
        return
    import torch

    from paper_2604_07644_b300 import build as B_
    from paper_2604_07644_b300 import native
    from paper_2604_07644_b300 import learned
    from paper_2604_07644_b300 import workloads as W
    from paper_2604_07644_b300.api import QPBatch

    assert torch.cuda.is_available(), "bench needs a CUDA device"
    torch.cuda.set_device(local)
    B_.build()
    native.load()
    dev = f"cuda:{local}"
    stream = torch.cuda.Stream(device=dev)
    prec = {"fp32": native.GPUSLS_FP32, "fp64": native.GPUSLS_FP64, "mixed": native.GPUSLS_MIXED}[args.precision]
    esz = 8 if prec == native.GPUSLS_FP64 else 4
    fam = W.family(0)
    base = 100000 + rank * args.batch
    qps = [fam.instance(base + i) for i in range(args.batch)]
    nx, nu, N, nc, nf = qps[0].dims()
    settings = native.default_settings(precision=prec, cluster=args.cluster, max_refine=3,
                                       fallback_iters=args.fallback, max_iter=6000, eps=EPS_IN, eps_kkt=EPS_KKT,
                                       check_every=CHECK_EVERY, sigma=SIGMA,
                                       eps_floor=1e-7 if prec == native.GPUSLS_FP64 else 1e-5,
                                       schedule=0 if args.index_order else 1)
    tuned = None
    if not args.no_autotune:
        from paper_2604_07644_b300 import autotune
        cache = autotune.Cache()
        settings, tuned = autotune.choose(qps, settings, expected_iters=250, tail_iters=2000, cache=cache)
    with torch.cuda.stream(stream):
        hb = QPBatch(qps, settings, stream=stream, device=dev)
        mlp = learned.load(args.model, max_batch=args.batch, stream=stream)
        heads = [(mlp, list(range(args.batch)), N)]   # features computed from the data inside the step
        g_learned = None if args.eager else hb.graph(heads=heads)
        g_cold = None if args.eager else hb.graph()

    def step_learned():
        if g_learned is not None:
            return g_learned.launch(stream)
        hb.reset()
        hb.warm_start_heads(heads)
        return hb.solve(fetch=False)

    def step_cold():
        if g_cold is not None:
            return g_cold.launch(stream)
        hb.reset()
        return hb.solve(fetch=False)

    def timed(fn, steps):
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            barrier(ws)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
        barrier(ws)
        return max_over_ranks(ws, e0.elapsed_time(e1))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step_learned()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_ms = timed(step_learned, args.steps)
    ms_per_step = t_ms / args.steps
    value = t_ms / (args.steps * args.batch * ws)

    def read_info(warm: bool):
        g = g_learned if warm else g_cold
        if g is not None:
            g.launch(stream)
            stream.synchronize()
            from types import SimpleNamespace
            return [SimpleNamespace(**d) for d in g.info()]
        info = (native.qp_info * args.batch)()
        hb.reset()
        if warm:
            hb.warm_start_heads(heads)
        hb.lib.qp_solve(hb.h, C_ptr(hb.x0), 0, 0.0, C_ptr(hb.out_x), C_ptr(hb.out_u), C_ptr(hb.out_l), info)
        return [info[i] for i in range(args.batch)]

    inf_w = read_info(True)
    sol_w = (hb.out_x.cpu().numpy(), hb.out_u.cpu().numpy())
    iters = [i.iters for i in inf_w]
    refs = [i.refactors for i in inf_w]
    kkts = [i.kkt for i in inf_w]
    stats = [i.status for i in inf_w]
    # the same batch solved cold (no learned warm start)
    with torch.cuda.stream(stream):
        step_cold()
    t_cold = timed(step_cold, max(1, args.steps))
    cold_ms = t_cold / (max(1, args.steps) * args.batch * ws)
    inf_c = read_info(False)

    # the same learned step with the factorization's block products on the
    # tensor cores (GPUSLS_MIXED: three TF32 passes, per-stage solves to FP64 accuracy)
    mixed = None
    if prec == native.GPUSLS_FP32:
        sm = native.default_settings(precision=native.GPUSLS_MIXED, cluster=int(settings.cluster),
                                     occupancy=int(settings.occupancy), max_refine=3, fallback_iters=args.fallback,
                                     max_iter=6000, eps_floor=1e-5, eps=EPS_IN, eps_kkt=EPS_KKT,
                                     check_every=CHECK_EVERY, sigma=SIGMA,
                                     schedule=0 if args.index_order else 1)
        with torch.cuda.stream(stream):
            hm = QPBatch(qps, sm, stream=stream, device=dev, pools=hb.pools)
            gm = hm.graph(heads=heads)
            for _ in range(2):
                gm.launch(stream)
        tm = timed(lambda: gm.launch(stream), max(1, args.steps))
        im = gm.info()
        xm, um = split_solution((hm.out_x.cpu().numpy(), hm.out_u.cpu().numpy()), qps)
        dm, _ = exact_distance(xm, um, len(qps))
        mixed = {"ms_per_qp": tm / (max(1, args.steps) * args.batch * ws),
                 "iters_mean": float(np.mean([i["iters"] for i in im])),
                 "kkt_max": float(np.max([i["kkt"] for i in im])),
                 "all_converged": all(i["status"] == 0 for i in im),
                 "max_rel_diff_vs_exact": dm,
                 "mode": "GPUSLS_MIXED: blocked-factorization block products in three TF32 passes (mma.sync), "
                         "per-stage solves to FP64 accuracy (FP32 inverse + Newton-Schulz step with an FP64 residual), "
                         "FP64 KKT gate"}
        gm.close()
        hm.close()

    # plain FP64 single-QP solves (cold, one QP per launch)
    plain = []
    for i in range(args.plain_qps):
        hp = QPBatch([qps[i]], native.default_settings(precision=native.GPUSLS_FP64, cluster=args.cluster,
                                                       eps=EPS_IN, eps_kkt=EPS_KKT, check_every=CHECK_EVERY,
                                                       sigma=SIGMA),
                     stream=stream, device=dev)
        with torch.cuda.stream(stream):
            hp.reset()
            hp.solve(fetch=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            hp.reset()
            e0.record(stream)
            hp.solve(fetch=False)
            e1.record(stream)
            torch.cuda.synchronize()
        plain.append(e0.elapsed_time(e1))
        hp.close()
    plain_ms = float(np.mean(plain)) if plain else None

    # end to end through the public API, every step: H2D of the problem data,
    # x0 and features from pinned memory, qp_update, learned warm start +
    # solve, D2H of (dx, du, lam).  The H2D of step k+1 runs on a copy stream
    # into a second set of device buffers while step k computes.
    e2e = None
    if not args.no_e2e:
        keys = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi")
        host = {k: hb.pools[k].cpu().pin_memory() for k in keys}
        host_x0 = hb.x0.cpu().pin_memory()
        bufs = [{k: torch.empty_like(hb.pools[k]) for k in keys} for _ in range(2)]
        x0b = [torch.empty_like(hb.x0) for _ in range(2)]
        out_host = [torch.empty_like(t, device="cpu").pin_memory() for t in (hb.out_x, hb.out_u, hb.out_l)]
        h2d = sum(t.numel() * 8 for t in host.values()) + host_x0.numel() * 8
        d2h = sum(t.numel() * 8 for t in out_host)
        copy_stream = torch.cuda.Stream(device=dev)

        def e2e_run(nsteps):
            ev_h2d = [None, None]
            ev_free = [None, None]   # buffer j consumed by its step's qp_update

            def issue_h2d(j):
                with torch.cuda.stream(copy_stream):
                    if ev_free[j] is not None:
                        copy_stream.wait_event(ev_free[j])
                    for k in keys:
                        bufs[j][k].copy_(host[k], non_blocking=True)
                    x0b[j].copy_(host_x0, non_blocking=True)
                    ev_h2d[j] = torch.cuda.Event()
                    ev_h2d[j].record(copy_stream)

            issue_h2d(0)
            for i in range(nsteps):
                j = i % 2
                if i + 1 < nsteps:
                    issue_h2d(1 - j)
                with torch.cuda.stream(stream):
                    stream.wait_event(ev_h2d[j])
                    hb.x0.copy_(x0b[j])
                    hb.update_pools(bufs[j])
                    ev_free[j] = torch.cuda.Event()
                    ev_free[j].record(stream)
                    step_learned()
                    for o, d in zip(out_host, (hb.out_x, hb.out_u, hb.out_l)):
                        o.copy_(d, non_blocking=True)

        with torch.cuda.stream(stream):
            e2e_run(2)
            torch.cuda.synchronize()
        barrier(ws)
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            copy_stream.wait_event(e0)
            e2e_run(args.steps)
            ej = torch.cuda.Event()
            ej.record(copy_stream)
            stream.wait_event(ej)
            e1.record(stream)
            torch.cuda.synchronize()
        barrier(ws)
        te = max_over_ranks(ws, e0.elapsed_time(e1))
        e2e = {"value": te / (args.steps * args.batch * ws), "unit": "ms/QP", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "overlap": "the H2D of step k+1 runs on a copy stream while step k computes"}

    # ---- further workloads of the same library (rank 0): the serving mix, the
    # humanoid-shaped QP, the humanoid SLS solve; solution checks ----
    cpu = None
    oracle_sols = []
    if rank == 0 and ws == 1 and args.cpu_sample > 0:
        n_s = min(args.cpu_sample, args.batch)
        ms_cpu, procs, oracle_sols = cpu_oracle_pool([base + i for i in range(n_s)])
        it_cpu = [r[1] for r in oracle_sols]
        cpu = {"value": ms_cpu, "unit": "ms/QP", "cores": procs, "kind": "oracle", "host": host_cpu(),
               "sample": f"the first {n_s} QPs of this batch, FP64 oracle ADMM to the 1e-4 KKT tolerance, one QP "
                         f"per worker process over {procs} cores; value = wall time / QPs; "
                         f"mean iters {np.mean(it_cpu):.0f}"}
    extra = {}
    # the further workloads once, in the single-GPU run (a scaling run holds
    # every GPU while rank 0 works)
    if rank == 0 and ws == 1 and not args.no_extras:
        extra = extra_workloads(args, qps, sol_w, stream, dev, oracle_sols)

    pk, pk_kind = peaks()
    algo = algorithmic_bytes_per_iter(nx, nu, N, nc, esz) * float(np.sum(iters))
    achieved = algo / (ms_per_step * 1e-3) / 1e9
    # DRAM bytes per QP-iteration of qp_kernel<float> from the ncu capture of the
    # iteration-only case at full occupancy (profiles/qp_kernel_iter_quadruped61_b45.md), scaled
    # by this launch's QP-iterations; must be re-measured when the kernel changes
    traffic = TRAFFIC_PER_QP_ITER * float(np.sum(iters)) if esz == 4 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
            "kernel": "qp_kernel (persistent cluster solve)", "peak_kind": pk_kind,
            "algorithmic_bytes_per_launch": algo}


    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "ms/QP", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if esz == 4 else "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "solver": "learned warm start + batched persistent GPU solve",
                           "batch": args.batch, "precision": args.precision,
                           "cluster": int(settings.cluster), "occupancy": int(settings.occupancy),
                           "launch_shape": ("autotuned" if tuned is not None else "fixed"),
                           "step": "eager calls" if args.eager else "one CUDA graph per step",
                           "launch_order": ("index" if args.index_order else
                                            "longest expected first (each QP's previous solve)"),
                           "parallelism": f"replicas x{ws}",
                           "l2": "inputs larger than L2 (FP64 pools 2.2 GB per 256 QPs)",
                           "model": os.path.basename(args.model)},
                "batched_cold_ms_per_qp": cold_ms,
                "mixed_precision": mixed,
                "plain_fp64_ms_per_qp": plain_ms,
                "iters_mean": float(np.mean(iters)), "iters_mean_cold": float(np.mean([i.iters for i in inf_c])),
                "refactors_mean": float(np.mean(refs)),
                "refactors_mean_cold": float(np.mean([i.refactors for i in inf_c])),
                "kkt_max": float(np.max(kkts)), "all_converged": all(s_ == 0 for s_ in stats),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": None if g_learned is None else g_learned.kernel_count() * args.steps,
                "clocks": clk.summary()}
        line.update(extra)
        print(json.dumps(line), flush=True)
    hb.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def C_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


if __name__ == "__main__":
    main()
