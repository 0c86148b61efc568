"""Train the warm-start network for the quadruped-shaped QP family on the GPU.

    python -m paper_2604_07644_b300.train_warmstart [--n 10000] [--epochs 120] [--out PATH]

Generates n family instances (indices 0..n-1), solves them cold with the plain
batched solver, trains the 2x256 MLP with the library's kernels and saves the
weights and normalization to PATH (default: warmstart_quadruped61.npz beside
this file).  Held-out evaluation instances use indices >= 100000.
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from . import build, learned, native
from . import workloads as W
from .api import MLP

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "warmstart_quadruped61.npz")


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=10000)
    p.add_argument("--epochs", type=int, default=120)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--out", default=DEFAULT_OUT)
    a = p.parse_args()
    build.build()
    native.load()
    fam = W.family(0)
    t0 = time.time()
    X, T, info = learned.generate(fam, list(range(a.n)))
    t1 = time.time()
    print(f"data: {len(X)} converged solves in {t1 - t0:.1f}s, mean iters {info['iters_mean']:.1f}", flush=True)
    mlp = MLP(X.shape[1], learned.HIDDEN, T.shape[1], max_batch=512)
    mlp.set_params(W.mlp_init(X.shape[1], learned.HIDDEN, T.shape[1], 0))
    losses = learned.train(mlp, X, T, epochs=a.epochs, lr=a.lr)
    t2 = time.time()
    print(f"training: {a.epochs} epochs in {t2 - t1:.1f}s, final loss {losses[-1]:.4f}", flush=True)
    learned.save(a.out, mlp, {"n": int(len(X)), "epochs": a.epochs, "lr": a.lr, "final_loss": float(losses[-1]),
                              "family_seed": 0, "data_iters_mean": info["iters_mean"]})
    print("saved", a.out)


if __name__ == "__main__":
    main()
