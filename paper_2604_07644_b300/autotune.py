"""Launch-shape autotuner for the batched persistent solve.

The solve kernel has two launch-shape knobs: the cluster size (CTAs per QP,
which sets the chunk of stages each CTA scans: ceil(N / cluster)) and the
occupancy (two CTAs per SM when they fit, or one CTA per SM with all of its
shared memory and issue slots).  Which is fastest depends on the state
dimension, the horizon and the batch size, so the tuner measures the
candidates on the caller's own problems and caches the winner per bucket:

    key = (device name, precision, nx bucket, N bucket, batch bucket)
    nx buckets 16 / 32 / 64 / 80, N buckets 32 / 64 / 128 / 256 / 1024 / 4096,
    batch buckets 1 / 8 / 64 / 256 / 4096.

A candidate is scored by the modeled time of one batched solve, per QP:

    max( T_batch(expected_iters),  T_one(tail_iters) ) / batch,

where T(k) = t(k1) + (k - k1) (t(k2) - t(k1)) / (k2 - k1) is the straight line
through two fixed-iteration timings (k1 < k2 iterations, so the factorization
and the per-iteration cost are both weighed), T_batch is timed on the whole
sample batch (throughput: every QP at the mean iteration count) and T_one on
its first QP alone (latency: the slowest QP of a batch, at tail_iters, bounds
the batch's makespan however well the rest is packed).  All timing is done
with CUDA events on the handle's stream; the tuner does no arithmetic of the
method.
"""
from __future__ import annotations

import copy
import json
import os
from dataclasses import dataclass

NX_BUCKETS = (16, 32, 64, 80)
N_BUCKETS = (32, 64, 128, 256, 1024, 4096)
B_BUCKETS = (1, 8, 64, 256, 4096)
# Every cluster size: a GPC holds two CTAs per SM, and the sizes that tile
# its slots best (6 on B300: four 8-CTA clusters leave slots idle) can beat
# the longer chains they imply.
CLUSTERS = (1, 2, 3, 4, 5, 6, 7, 8)
OCCUPANCIES = (0, 1)


def bucket(v: int, edges) -> int:
    """Smallest edge >= v (the last edge for anything larger)."""
    for e in edges:
        if v <= e:
            return e
    return edges[-1]


def key(device: str, precision: int, nx: int, N: int, batch: int) -> str:
    return f"{device}|p{precision}|nx{bucket(nx, NX_BUCKETS)}|N{bucket(N, N_BUCKETS)}|B{bucket(batch, B_BUCKETS)}"


def candidates(N: int) -> list[tuple[int, int]]:
    """(cluster, occupancy) pairs worth trying for horizon N: a cluster larger
    than N would leave CTAs without stages."""
    return [(c, o) for c in CLUSTERS if c <= max(1, N) for o in OCCUPANCIES]


def score(t1: float, t2: float, k1: int, k2: int, expected_iters: float) -> float:
    """Modeled solve time from two fixed-iteration timings t(k1), t(k2)."""
    slope = (t2 - t1) / float(k2 - k1)
    return (t1 - k1 * slope) + expected_iters * slope


def makespan(batch_t: tuple[float, float], one_t: tuple[float, float], k1: int, k2: int, expected_iters: float,
             tail_iters: float) -> float:
    """Modeled time of one batched solve: throughput of the batch at the mean
    iteration count, or the latency of one QP at the tail count, whichever is
    longer."""
    return max(score(batch_t[0], batch_t[1], k1, k2, expected_iters),
               score(one_t[0], one_t[1], k1, k2, tail_iters))


@dataclass
class Choice:
    cluster: int
    occupancy: int
    ms_per_qp: float


class Cache:
    """JSON cache of tuned choices; path from GPUSLS_TUNE_CACHE, else under
    the user's cache directory."""

    def __init__(self, path: str | None = None):
        self.path = path or os.environ.get("GPUSLS_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "gpusls", "autotune.json")
        self.data = {}
        try:
            with open(self.path) as f:
                self.data = json.load(f)
        except (OSError, ValueError):
            self.data = {}

    def get(self, k: str) -> Choice | None:
        v = self.data.get(k)
        return Choice(**v) if v else None

    def put(self, k: str, c: Choice):
        self.data[k] = dict(cluster=c.cluster, occupancy=c.occupancy, ms_per_qp=c.ms_per_qp)
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except OSError:
            pass


def _timer(qps, settings, pools=None):
    """A handle over qps that runs exactly k iterations per solve (no stop
    test, fixed rho), and a function timing one reset + solve of k iterations
    (best of two, after one warm-up)."""
    import torch

    from .api import QPBatch, _dptr
    s = copy.copy(settings)
    s.fixed_iters = 0
    s.sigma = 0
    s.eps = 0.0
    s.eps_kkt = 0.0
    stream = torch.cuda.Stream()
    qb = QPBatch(qps, s, stream=stream, pools=pools)

    def run(k: int) -> float:
        from . import native
        info = (native.qp_info * qb.B)()

        def once():
            qb.reset()
            qb.lib.qp_solve(qb.h, _dptr(qb.x0), int(k), 0.0, _dptr(qb.out_x), _dptr(qb.out_u), _dptr(qb.out_l),
                            info)

        with torch.cuda.stream(stream):
            once()
            best = float("inf")
            for _ in range(2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                once()
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
        return best

    return qb, run


def tune(qps, settings, expected_iters: float = 250.0, tail_iters: float | None = None, k1: int = 10, k2: int = 40,
         cache: Cache | None = None, sample: int = 0) -> Choice:
    """Measure every candidate launch shape on `qps` (or the first `sample` of
    them) and return (and cache) the fastest for their bucket.  tail_iters
    (default 8 x expected_iters) is the iteration count of the slowest QP."""
    tail = 8.0 * expected_iters if tail_iters is None else float(tail_iters)
    import torch

    qps = list(qps)
    if sample and len(qps) > sample:
        qps = qps[:sample]
    nx = max(q.nx for q in qps)
    N = max(q.N for q in qps)
    dev = torch.cuda.get_device_name()
    k = key(dev, settings.precision, nx, N, len(qps))
    best = None
    pools = None
    for c, o in candidates(N):
        s = copy.copy(settings)
        s.cluster = c
        s.occupancy = o
        try:
            qb, run = _timer(qps, s, pools)
            pools = qb.pools
            bt = (run(k1), run(k2))
            qb.close()
            q1, run1 = _timer(qps[:1], s)
            ot = (run1(k1), run1(k2))
            q1.close()
        except RuntimeError:
            continue                               # shape does not fit (shared memory)
        ms = makespan(bt, ot, k1, k2, expected_iters, tail) / len(qps)
        # ties (within 2 %) go to the larger cluster: lower latency per QP
        if best is None or ms < 0.98 * best.ms_per_qp or (ms <= 1.02 * best.ms_per_qp and c > best.cluster):
            best = Choice(c, o, ms)
    if best is None:
        raise RuntimeError("autotune: no candidate launch shape fits these problems")
    if cache is not None:
        cache.put(k, best)
    return best


def choose(qps, settings, expected_iters: float = 250.0, tail_iters: float | None = None, cache: Cache | None = None,
           sample: int = 0):
    """Settings with the tuned cluster size and occupancy for `qps`, from the
    cache when the bucket was tuned before, else by measuring."""
    import torch

    cache = cache if cache is not None else Cache()
    qps = list(qps)
    nx = max(q.nx for q in qps)
    N = max(q.N for q in qps)
    k = key(torch.cuda.get_device_name(), settings.precision, nx, N, len(qps))
    c = cache.get(k)
    if c is None:
        c = tune(qps, settings, expected_iters=expected_iters, tail_iters=tail_iters, cache=cache, sample=sample)
    s = copy.copy(settings)
    s.cluster = c.cluster
    s.occupancy = c.occupancy
    return s, c
