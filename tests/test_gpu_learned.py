"""What the trained warm-start network gains over the method without it, on
held-out instances of the quadruped-shaped QP family (the network was trained
on instances 0..9999; these are 100000+), and that a warm start that fails
falls back to the cold method."""
import os

import numpy as np
import pytest
import torch

from oracle import kkt
from paper_2604_07644_b300 import native
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu

MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2604_07644_b300",
                     "warmstart_quadruped61.npz")


def test_learned_warm_start_gain(lib):
    from paper_2604_07644_b300 import learned
    from paper_2604_07644_b300.api import QPBatch
    fam = W.family(0)
    qps = [fam.instance(100000 + 500 + i) for i in range(64)]
    s = native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, max_refine=3, fallback_iters=1500)
    qb = QPBatch(qps, s)
    cold = qb.solve()
    mlp = learned.load(MODEL, max_batch=64)
    qb.reset()
    mlp.warm_start(qb, torch.from_numpy(learned.features(qps)).cuda())
    warm = qb.solve()
    assert all(i["status"] == native.GPUSLS_OK for i in warm.info)
    ic = np.mean([i["iters"] for i in cold.info])
    iw = np.mean([i["iters"] for i in warm.info])
    rc = np.mean([i["refactors"] for i in cold.info])
    rw = np.mean([i["refactors"] for i in warm.info])
    print(f"held-out 64: iterations cold {ic:.1f} warm {iw:.1f}; refactors cold {rc:.2f} warm {rw:.2f}")
    assert iw < 0.95 * ic
    assert rw < 0.75 * rc
    for i in range(0, 64, 16):
        assert kkt.kkt_residual(qps[i], warm.dx[i], warm.du[i], warm.lam[i]) <= 1.0001e-4
    mlp.close()
    qb.close()


def test_bad_warm_start_falls_back_to_cold(lib):
    """A deliberately wrong warm start (huge multipliers, rho at its upper
    clamp) that has not converged by fallback_iters restarts cold and still
    returns the cold solution."""
    from paper_2604_07644_b300.api import QPBatch
    fam = W.family(0)
    qp = fam.instance(100777)
    s = native.default_settings(precision=native.GPUSLS_FP32, eps_floor=1e-5, fallback_iters=50)
    qb = QPBatch([qp], s)
    cold = qb.solve()
    qb.reset()
    qb.set_warm_start([np.full(qp.m, 3.0)], [np.full(qp.m, 50.0)], 5e3)
    r = qb.solve()
    assert r.info[0]["status"] == native.GPUSLS_OK
    assert np.max(np.abs(r.dx[0] - cold.dx[0])) < 1e-3
    qb.close()
