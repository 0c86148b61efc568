"""Golden fixtures (tests/golden/, written by make_golden.py from the oracle
alone): the oracle still reproduces them, and the GPU path matches them."""
import json
import os

import numpy as np
import pytest

from oracle import activeset, admm
from oracle import sls as osls
from paper_2604_07644_b300 import workloads as W

G = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(G, name)) as f:
        return json.load(f)


def test_oracle_reproduces_tiny_bruteforce():
    for c in load("tiny_bruteforce.json")["cases"]:
        x, u, lam, _ = activeset.brute_force(W.tiny(c["seed"]))
        assert np.allclose(x, c["x"], atol=1e-12) and np.allclose(u, c["u"], atol=1e-12)


def test_oracle_reproduces_plain4d_iterates():
    g = load("plain4d_admm9.json")
    r = admm.admm(W.plain_4d(0), admm.Settings(rho0=0.3, sigma=0), iters=9)
    assert np.allclose(r.x, g["x"], atol=1e-12) and np.allclose(r.lam, g["lam"], atol=1e-12)


def test_oracle_reproduces_sls_small():
    g = load("sls_small.json")
    Px, Pu, h, hf, _ = osls.solve(W.sls_small(0))
    assert np.allclose(Px, g["Phi_x"], atol=1e-12) and np.allclose(h, g["h"], atol=1e-12)


@pytest.mark.gpu
def test_gpu_matches_golden(lib):
    from paper_2604_07644_b300 import native
    from paper_2604_07644_b300.api import SLS, QPBatch
    for c in load("tiny_bruteforce.json")["cases"]:
        qb = QPBatch([W.tiny(c["seed"])], native.default_settings(precision=native.GPUSLS_FP64, eps=1e-10,
                                                                     eps_kkt=1e-9, max_iter=100000))
        r = qb.solve()
        assert np.max(np.abs(r.dx[0] - np.array(c["x"]))) < 1e-6
        qb.close()
    g = load("plain4d_admm9.json")
    qb = QPBatch([W.plain_4d(0)], native.default_settings(precision=native.GPUSLS_FP64, sigma=0, fixed_iters=9),
                 rho=0.3)
    r = qb.solve()
    assert np.max(np.abs(r.dx[0] - np.array(g["x"]))) < 1e-9 * max(1.0, np.max(np.abs(g["x"])))
    qb.close()
    g = load("sls_small.json")
    sp = W.sls_small(0)
    s = SLS(sp.nx, sp.nu, sp.N, sp.nc, sp.nf, per_j_tau=sp.tau is not None, precision=native.GPUSLS_FP64)
    Px, Pu, h, hf = s.solve(sp)
    assert np.max(np.abs(Px - np.array(g["Phi_x"]))) < 1e-9 and np.max(np.abs(h - np.array(g["h"]))) < 1e-9
    s.close()
