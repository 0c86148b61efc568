"""Writes tests/golden/exact_quadruped61.npz from the FP64 oracle alone.

    python tests/golden/make_exact.py [--procs P]

The stored values are the exact optima of eq. sqp_qp for eight held-out
instances of the quadruped-shaped family (nx=61, nu=12, N=100, nc=20, nf=8;
instances 100000 + i for the listed i, the first QPs of the benchmark batch
plus its two slowest), found by oracle.admm.exact_solution: ADMM driven to a
1e-11 tolerance, then a dense-KKT solve on the detected active set.  No GPU
code is imported.  One instance takes about a minute of CPU time (the dense
KKT system has ~13.5 K rows), so the instances run in a process pool.

Fields: ids [8], x [8, N+1, nx], u [8, N, nu], lam [8, N nc + nf], kkt [8]
(the oracle's own KKT residual of each stored optimum).
"""
import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

IDS = [0, 1, 2, 3, 46, 128, 210, 255]
OUT = os.path.join(HERE, "exact_quadruped61.npz")


def solve_one(i):
    sys.path.insert(0, ROOT)
    from oracle import admm, kkt
    from paper_2604_07644_b300 import workloads as W
    qp = W.family(0).instance(100000 + i)
    x, u, lam = admm.exact_solution(qp)
    return i, x, u, lam, kkt.kkt_residual(qp, x, u, lam)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=min(len(IDS), os.cpu_count() or 1))
    a = ap.parse_args()
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = sorted(pool.map(solve_one, IDS))
    np.savez_compressed(OUT, ids=np.array(IDS), x=np.stack([r[1] for r in res]), u=np.stack([r[2] for r in res]),
                        lam=np.stack([r[3] for r in res]), kkt=np.array([r[4] for r in res]))
    print("kkt of the stored optima:", [f"{r[4]:.1e}" for r in res])


if __name__ == "__main__":
    main()
