"""Train the warm-start networks on the GPU with the library's kernels.

    python -m paper_2604_07644_b300.train_warmstart [--which headline|mix|all] [--n 10000] [--epochs 120]

headline: the quadruped-shaped family (nx=61, nu=12, N=100; instances
  0..n-1) -> warmstart_quadruped61.npz.
mix: one network per shape family of the serving mix (12D/4 quadrotor-
  shaped, 61D/12 and 75D/21 legged; horizons N ~ U{16..128} per instance,
  outputs laid out for 128 stages) -> warmstart_mix12/61/75.npz.
Every network sees the library's linearization features (qp_features) of
its QP; its targets are the converged ADMM state (z, lambda, log rho) of
cold solves by the plain batched solver.  Held-out evaluation instances use
indices >= 100000.
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


def fit(X, T, epochs, lr, out, meta, half):
    mlp = MLP(X.shape[1], learned.HIDDEN, T.shape[1], max_batch=512)
    mlp.set_params(W.mlp_init(X.shape[1], learned.HIDDEN, T.shape[1], 0))
    t0 = time.time()
    losses = learned.train(mlp, X, T, epochs=epochs, lr=lr)
    print(f"training: {epochs} epochs in {time.time() - t0:.1f}s, final loss {losses[-1]:.4f}", flush=True)
    learned.save(out, mlp, dict(meta, epochs=epochs, lr=lr, final_loss=float(losses[-1])), half=half)
    mlp.close()
    print("saved", out, flush=True)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--which", default="all", choices=["headline", "mix", "all"])
    p.add_argument("--n", type=int, default=10000)
    p.add_argument("--epochs", type=int, default=120)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--out-dir", default=HERE)
    a = p.parse_args()
    build.build()
    native.load()
    if a.which in ("headline", "all"):
        t0 = time.time()
        X, T, info = learned.generate_family(W.family(0), list(range(a.n)))
        print(f"headline data: {len(X)} solves in {time.time() - t0:.1f}s, mean iters {info['iters_mean']:.1f}")
        fit(X, T, a.epochs, a.lr, os.path.join(a.out_dir, "warmstart_quadruped61.npz"),
            {"n": int(len(X)), "family": "family(0) 61/12/100", "features": "qp_features",
             "data_iters_mean": info["iters_mean"]}, half=False)
    if a.which in ("mix", "all"):
        for kind, name in enumerate(learned.MIX_MODELS):
            fam = W.mix_family(kind)
            Ns = [int(v) for v in W.rng(24, kind).integers(16, W.MIX_N_MAX + 1, a.n)]
            t0 = time.time()
            X, T, info = learned.generate_family(fam, list(range(a.n)), Ns, n_stage=W.MIX_N_MAX)
            print(f"mix family {kind} data: {len(X)} solves in {time.time() - t0:.1f}s, "
                  f"mean iters {info['iters_mean']:.1f}")
            fit(X, T, a.epochs, a.lr, os.path.join(a.out_dir, name),
                {"n": int(len(X)), "family": f"mix_family({kind})", "n_stage": W.MIX_N_MAX,
                 "features": "qp_features", "data_iters_mean": info["iters_mean"]}, half=True)


if __name__ == "__main__":
    main()
