"""Learned ADMM warm start: training data from the plain solver, training of
the warm-start network on the GPU, and warm-started batched solves.

Only orchestration lives here; every arithmetic step runs in the library's
kernels (ADMM solves, MLP forward/backward/Adam, normalization, warm-start
assembly).
"""
from __future__ import annotations

import numpy as np
import torch

from . import native
from .api import MLP, QPBatch, pool

HIDDEN = 256


def features(qps) -> np.ndarray:
    """Network inputs: the initial state x0 and the linearization parameters
    theta of each instance (float32 [B][nx + n_theta])."""
    return np.stack([np.asarray(q.features, dtype=np.float32) for q in qps])


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


def save(path: str, mlp: MLP, meta: dict):
    params = mlp.get_params()
    norm = mlp.get_normalization()
    np.savez_compressed(path, W1=params[0], b1=params[1], W2=params[2], b2=params[3], W3=params[4], b3=params[5],
                        xm=norm[0], xs=norm[1], ym=norm[2], ys=norm[3],
                        meta=np.array(repr(meta)))


def load(path: str, max_batch: int, stream=None) -> MLP:
    d = np.load(path)
    n_in, n_out, hid = d["W1"].shape[1], d["W3"].shape[0], d["W1"].shape[0]
    m = MLP(n_in, hid, n_out, max_batch=max_batch, stream=stream)
    m.set_params([d["W1"], d["b1"], d["W2"], d["b2"], d["W3"], d["b3"]])
    m.set_normalization(d["xm"], d["xs"], d["ym"], d["ys"])
    return m
