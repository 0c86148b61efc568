"""GPU parity of the warm-start MLP kernels against the FP64 oracle evaluated
with the same BF16 operand rounding (oracle.mlp, bf16=True).

Tolerance: BF16 operands carry a relative rounding of 2^-8; an FP32-versus-FP64
difference in an activation can flip one operand's rounding (one BF16 ulp), so
results are compared to 2e-2 of the largest magnitude (outputs 1e-2)."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2604_07644_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-30, float(np.max(np.abs(b)))))


def make(n_in, hid, n_out, B, seed):
    from paper_2604_07644_b300.api import MLP
    params = W.mlp_init(n_in, hid, n_out, seed)
    g = np.random.default_rng(seed)
    params[1] = 0.1 * g.standard_normal(hid)
    params[3] = 0.1 * g.standard_normal(hid)
    params[5] = 0.1 * g.standard_normal(n_out)
    params = [p.astype(np.float32).astype(np.float64) for p in params]
    X = g.standard_normal((B, n_in)).astype(np.float32).astype(np.float64)
    T = g.standard_normal((B, n_out)).astype(np.float32).astype(np.float64)
    m = MLP(n_in, hid, n_out, max_batch=B)
    m.set_params(params)
    return m, params, X, T


@pytest.mark.parametrize("dims", [(5, 16, 3, 8), (69, 256, 4017, 64), (37, 96, 200, 130)])
def test_forward_matches_oracle(lib, dims):
    n_in, hid, n_out, B = dims
    m, params, X, T = make(n_in, hid, n_out, B, 1)
    Y = m.forward(torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy()
    Yo, _ = omlp.forward(params, X, bf16=True)
    assert rel(Y, Yo) < 1e-2
    m.close()


@pytest.mark.parametrize("dims", [(5, 16, 3, 8), (69, 256, 4017, 64), (37, 96, 200, 130)])
def test_gradients_match_oracle(lib, dims):
    n_in, hid, n_out, B = dims
    m, params, X, T = make(n_in, hid, n_out, B, 2)
    grads, loss = m.gradients(torch.from_numpy(X.astype(np.float32)).cuda(),
                              torch.from_numpy(T.astype(np.float32)).cuda())
    og = omlp.backward(params, X, T, bf16=True)
    for gg, oo in zip(grads, og):
        assert rel(gg, oo) < 2e-2, rel(gg, oo)
    assert abs(loss - omlp.loss(params, X, T, bf16=True)) < 1e-2 * omlp.loss(params, X, T, bf16=True)
    m.close()


def test_adam_step_matches_oracle(lib):
    """One train step with identity normalization equals the oracle's Adam step
    on the oracle's gradients (first step: lr * sign(g) up to eps)."""
    n_in, hid, n_out, B = 6, 32, 5, 16
    m, params, X, T = make(n_in, hid, n_out, B, 3)
    lr = 1e-3
    m.train_step(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T.astype(np.float32)).cuda(), lr)
    newp = m.get_params()
    og = omlp.backward(params, X, T, bf16=True)
    mm = [np.zeros_like(p) for p in params]
    vv = [np.zeros_like(p) for p in params]
    op, _, _ = omlp.adam_step([p.copy() for p in params], og, mm, vv, 1, lr)
    for a, b, p in zip(newp, op, params):
        # Adam's first step moves each weight by ~lr*sign(g); where |g| is tiny the
        # sign can differ between FP32/BF16 and FP64, so compare the movement.
        moved = np.abs(a - p)
        assert np.all(moved <= lr * 1.01 + 1e-7)
        agree = np.mean(np.sign(a - p) == np.sign(b - p))
        assert agree > 0.9
    m.close()


def test_training_reduces_loss(lib):
    from paper_2604_07644_b300.api import MLP
    g = np.random.default_rng(0)
    n_in, hid, n_out, B = 8, 64, 4, 256
    X = g.standard_normal((B, n_in)).astype(np.float32)
    T = np.stack([X[:, 0] - X[:, 1], np.maximum(X[:, 2], 0), X[:, 3] * 0.5, np.abs(X[:, 4])], axis=1).astype(np.float32)
    m = MLP(n_in, hid, n_out, max_batch=B)
    m.set_params(W.mlp_init(n_in, hid, n_out, 4))
    Xt, Tt = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m.fit_normalization(Xt, Tt)
    l0 = m.train_step(Xt, Tt, 1e-3)
    for _ in range(300):
        l = m.train_step(Xt, Tt, 1e-3)
    assert l < 0.1 * l0
    m.close()


def test_save_and_load_round_trip(lib, tmp_path):
    """mlp_save writes parameters and normalization; mlp_load into a fresh
    handle of the same sizes reproduces the network bit for bit; a file of
    other sizes, a truncated or a foreign file is rejected with
    GPUSLS_ERR_INVALID and leaves the handle unchanged."""
    from paper_2604_07644_b300.api import MLP
    m, params, X, T = make(37, 96, 20, 16, 4)
    Xt = torch.from_numpy(X.astype(np.float32)).cuda()
    Tt = torch.from_numpy(T.astype(np.float32)).cuda()
    m.fit_normalization(Xt, Tt)
    y0 = m.forward(Xt).cpu().numpy()
    path = str(tmp_path / "net.bin")
    m.save(path)
    m2 = MLP(37, 96, 20, max_batch=16)
    m2.load(path)
    assert np.array_equal(m2.forward(Xt).cpu().numpy(), y0)
    other = MLP(37, 64, 20, max_batch=16)
    with pytest.raises(RuntimeError, match="failed with invalid"):
        other.load(path)
    raw = open(path, "rb").read()
    (tmp_path / "short.bin").write_bytes(raw[:-4])
    (tmp_path / "foreign.bin").write_bytes(b"NOTANMLP" + raw[8:])
    for bad in ("short.bin", "foreign.bin", "missing.bin"):
        with pytest.raises(RuntimeError, match="failed with invalid"):
            m2.load(str(tmp_path / bad))
    assert np.array_equal(m2.forward(Xt).cpu().numpy(), y0)
    for h in (m, m2, other):
        h.close()
