"""Learned ADMM warm start: training data from the plain solver, training of
the warm-start network on the GPU, and warm-started batched solves.

Only orchestration lives here; every arithmetic step runs in the library's
kernels (ADMM solves, MLP forward/backward/Adam, normalization, warm-start
assembly).
"""
from __future__ import annotations

import os

import numpy as np
import torch

from . import native
from .api import MLP, QPBatch, pool

HIDDEN = 256


def lin_features(qb: QPBatch, idx=None) -> np.ndarray:
    """Network inputs computed by the library from the data the caller gave
    the handle (qp_features): x0 and fixed projections of the linearization,
    float32 [count][nx + 4 GPUSLS_FEATURE_P + 1]."""
    return qb.features(idx).cpu().numpy()


def padded_targets(qb: QPBatch, res, n_stage: int) -> np.ndarray:
    """Targets (z, lambda, log rho) of solved QPs laid out for horizon n_stage
    (the qp_warm_start_heads layout): stage rows first, zero-padded past each
    QP's N, then the terminal rows (float32 [B][2 (n_stage nc + nf) + 1])."""
    z, y, rho = qb.get_state()
    rows = []
    for i, qp in enumerate(qb.qps):
        nc, nf, N = qp.nc, qp.nf, qp.N
        mmax = n_stage * nc + nf

        def place(v):
            out = np.zeros(mmax)
            out[:N * nc] = v[:N * nc]
            out[n_stage * nc:] = v[N * nc:]
            return out

        rows.append(np.concatenate([place(z[i]), place(res.lam[i]), [np.log(rho[i])]]).astype(np.float32))
    return np.stack(rows)


def generate_family(fam, indices, horizons=None, n_stage: int | None = None, chunk: int = 512,
                    precision=native.GPUSLS_FP32, log=print):
    """Solve family instances (indices, optional per-instance horizons) cold
    with the plain batched solver; return (X, T, info) for the converged ones,
    X from the library's features, T in the qp_warm_start_heads layout."""
    X, T, its = [], [], []
    for c0 in range(0, len(indices), chunk):
        ids = indices[c0:c0 + chunk]
        Ns = [None] * len(ids) if horizons is None else horizons[c0:c0 + chunk]
        qps = [fam.instance(i, N) for i, N in zip(ids, Ns)]
        ns = n_stage or max(q.N for q in qps)
        s = native.default_settings(precision=precision,
                                    eps_floor=1e-5 if precision != native.GPUSLS_FP64 else 1e-7)
        qb = QPBatch(qps, s)
        r = qb.solve()
        ok = [i for i, inf in enumerate(r.info) if inf["status"] == native.GPUSLS_OK]
        X.append(lin_features(qb)[ok])
        T.append(padded_targets(qb, r, ns)[ok])
        its += [r.info[i]["iters"] for i in ok]
        qb.close()
        log(f"  generated {c0 + len(qps)}/{len(indices)}: converged {len(ok)}/{len(qps)}, "
            f"mean iters {np.mean([inf['iters'] for inf in r.info]):.0f}")
    return np.concatenate(X), np.concatenate(T), {"iters_mean": float(np.mean(its))}


def solve_targets(qb: QPBatch, res) -> np.ndarray:
    """Training targets (z, lambda, log rho) of solved QPs (float32 [B][2m+1])."""
    z, y, rho = qb.get_state()
    rows = []
    for i in range(qb.B):
        rows.append(np.concatenate([z[i], res.lam[i], [np.log(rho[i])]]).astype(np.float32))
    return np.stack(rows)


def generate(fam, indices, chunk: int = 512, precision=native.GPUSLS_FP32, log=print):
    """Solve the family instances `indices` cold with the plain batched solver
    and return (X, T, info) for the converged ones."""
    X, T, its = [], [], []
    qb = None
    for c0 in range(0, len(indices), chunk):
        qps = [fam.instance(i) for i in indices[c0:c0 + chunk]]
        s = native.default_settings(precision=precision,
                                    eps_floor=1e-5 if precision == native.GPUSLS_FP32 else 1e-7)
        if qb is None or qb.B != len(qps):
            if qb is not None:
                qb.close()
            qb = QPBatch(qps, s)
        else:
            qb.qps = qps
            keys = ("A", "B", "c", "Q", "R", "S", "q", "r", "C", "D", "CN", "lo", "hi")
            qb.update_pools({k: pool([getattr(q, k) for q in qps]) for k in keys})
            qb.set_x0([q.x0 for q in qps])
            qb.reset()
        r = qb.solve()
        ok = [i for i, inf in enumerate(r.info) if inf["status"] == native.GPUSLS_OK]
        X.append(features([qps[i] for i in ok]))
        T.append(solve_targets(qb, r)[ok])
        its += [r.info[i]["iters"] for i in ok]
        log(f"  generated {c0 + len(qps)}/{len(indices)}: converged {len(ok)}/{len(qps)}, "
            f"mean iters {np.mean([inf['iters'] for inf in r.info]):.0f}")
    if qb is not None:
        qb.close()
    return np.concatenate(X), np.concatenate(T), {"iters_mean": float(np.mean(its))}


def train(mlp: MLP, X: np.ndarray, T: np.ndarray, epochs: int = 60, batch: int = 256, lr: float = 1e-3,
          seed: int = 0, log=print, lr_final: float | None = None, reshuffle: bool = False):
    """Minibatch Adam on (X, T).  Order: a fixed random permutation (rotated
    each epoch), or a fresh seeded permutation every epoch (reshuffle).  The
    step size decays from lr to lr_final on a cosine when lr_final is given."""
    import math
    g = np.random.Generator(np.random.Philox(seed))
    perm = g.permutation(len(X))
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(T[perm])).cuda()
    mlp.fit_normalization(Xd, Td)
    n = (len(X) // batch) * batch
    losses = []
    for ep in range(epochs):
        lr_e = lr if lr_final is None else lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * ep / epochs))
        if reshuffle and ep > 0:
            idx = torch.from_numpy(g.permutation(len(X))).cuda()
            Xe, Te, off = Xd[idx], Td[idx], 0
        else:
            Xe, Te, off = Xd, Td, (ep * 97) % batch
        tot = 0.0
        steps = 0
        for s in range(off, n - batch + 1, batch):
            tot += mlp.train_step(Xe[s:s + batch], Te[s:s + batch], lr_e)
            steps += 1
        losses.append(tot / max(1, steps))
        if log and (ep % 10 == 0 or ep == epochs - 1):
            log(f"  epoch {ep}: loss {losses[-1]:.4f} (lr {lr_e:.2e})")
    return losses


def save(path: str, mlp: MLP, meta: dict, half: bool = False):
    """Weights and normalization to an npz (half: weight matrices stored as
    float16, which the BF16 products of the network do not resolve anyway)."""
    params = mlp.get_params()
    norm = mlp.get_normalization()
    cast = (lambda a: a.astype(np.float16)) if half else (lambda a: a)
    np.savez_compressed(path, W1=cast(params[0]), b1=params[1], W2=cast(params[2]), b2=params[3],
                        W3=cast(params[4]), b3=params[5], xm=norm[0], xs=norm[1], ym=norm[2], ys=norm[3],
                        meta=np.array(repr(meta)))


def load(path: str, max_batch: int, stream=None) -> MLP:
    d = np.load(path)
    n_in, n_out, hid = d["W1"].shape[1], d["W3"].shape[0], d["W1"].shape[0]
    m = MLP(n_in, hid, n_out, max_batch=max_batch, stream=stream)
    m.set_params([np.asarray(d[k], dtype=np.float32) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    m.set_normalization(d["xm"], d["xs"], d["ym"], d["ys"])
    return m


MIX_MODELS = ("warmstart_mix12.npz", "warmstart_mix61.npz", "warmstart_mix75.npz")


def mix_heads(qps_kinds, model_dir: str, stream=None):
    """The per-family heads of the serving mix for a list of (QP, kind):
    [(MLP, QP indices, n_stage)] for QPBatch.graph(heads=...) /
    warm_start_heads, and the networks to close."""
    from . import workloads as W
    heads = []
    for k, name in enumerate(MIX_MODELS):
        ids = [i for i, (_, kind) in enumerate(qps_kinds) if kind == k]
        if ids:
            heads.append((load(os.path.join(model_dir, name), max_batch=max(1, len(ids)), stream=stream), ids,
                          W.MIX_N_MAX))
    return heads
