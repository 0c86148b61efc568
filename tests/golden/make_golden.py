"""Writes the golden fixtures of tests/golden/ from the FP64 oracle alone.

    python tests/golden/make_golden.py

Every stored value comes from oracle/ (no GPU code is imported); the inputs
come from the seeded generators.  The paper prints no numeric worked example,
so these fixtures pin the oracle against its own earlier output (a regression
check) and give the GPU tests fixed expected values:
  tiny_bruteforce.json   active-set brute-force optima of tiny LTV-QPs
                         (nx=2, nu=1, N=3), the exact solution of eq. sqp_qp
  plain4d_admm9.json     9 ADMM iterations (rho 0.3 fixed) on the 4D problem
  sls_small.json         Phi_x, Phi_u and margins of a small SLS problem
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import activeset, admm  # noqa: E402
from oracle import sls as osls  # noqa: E402
from paper_2604_07644_b300 import workloads as W  # noqa: E402


def _dump(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=1)


def main():
    cases = []
    for seed in range(4):
        qp = W.tiny(seed)
        x, u, lam, _ = activeset.brute_force(qp)
        cases.append({"seed": seed, "x": np.asarray(x).tolist(), "u": np.asarray(u).tolist(),
                      "lam": np.asarray(lam).tolist()})
    _dump("tiny_bruteforce.json", {"generator": "workloads.tiny(seed)", "solver": "oracle.activeset.brute_force",
                                   "cases": cases})
    qp = W.plain_4d(0)
    r = admm.admm(qp, admm.Settings(rho0=0.3, sigma=0), iters=9)
    _dump("plain4d_admm9.json", {"generator": "workloads.plain_4d(0)", "solver": "oracle.admm.admm, rho 0.3, "
                                 "sigma 0, 9 iterations", "x": r.x.tolist(), "u": r.u.tolist(),
                                 "lam": r.lam.tolist()})
    sp = W.sls_small(0)
    Px, Pu, h, hf, _ = osls.solve(sp)
    _dump("sls_small.json", {"generator": "workloads.sls_small(0)", "solver": "oracle.sls.solve",
                             "Phi_x": Px.tolist(), "Phi_u": Pu.tolist(), "h": h.tolist(), "hf": hf.tolist()})


if __name__ == "__main__":
    main()
