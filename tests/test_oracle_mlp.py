"""Pins of the oracle's MLP (the learned warm start has no paper counterpart)."""
import numpy as np
import pytest

from oracle import mlp
from paper_2604_07644_b300 import workloads as W


def _params(seed=0, n_in=5, hidden=7, n_out=3):
    p = W.mlp_init(n_in, hidden, n_out, seed)
    g = np.random.default_rng(seed)
    p[1] = 0.1 * g.standard_normal(p[1].shape)
    p[3] = 0.1 * g.standard_normal(p[3].shape)
    p[5] = 0.1 * g.standard_normal(p[5].shape)
    return p


def test_gradients_match_finite_differences():
    g = np.random.default_rng(3)
    params = _params()
    X = g.standard_normal((6, 5))
    T = g.standard_normal((6, 3))
    _, (X_, z1, h1, z2, h2) = mlp.forward(params, X)
    assert min(np.min(np.abs(z1)), np.min(np.abs(z2))) > 1e-4   # away from ReLU kinks
    grads = mlp.backward(params, X, T)
    h = 1e-6
    for pi in range(len(params)):
        flat = params[pi].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 9)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(params, X, T)
            flat[idx] = old - h
            lm = mlp.loss(params, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[pi].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd))


def test_one_hidden_unit_by_hand():
    """1-1-1-1 network, one sample, gradients worked out by hand."""
    w1, b1, w2, b2, w3, b3 = 0.5, 0.1, -1.5, 2.0, 0.8, -0.3
    x, t = 2.0, 1.0
    params = [np.array([[w1]]), np.array([b1]), np.array([[w2]]), np.array([b2]),
              np.array([[w3]]), np.array([b3])]
    z1 = w1 * x + b1             # 1.1
    h1 = z1                      # relu, positive
    z2 = w2 * h1 + b2            # 0.35
    h2 = z2
    y = w3 * h2 + b3             # -0.02
    dy = y - t                   # -1.02
    expect = [dy * w3 * w2 * x, dy * w3 * w2, dy * w3 * h1, dy * w3, dy * h2, dy]
    grads = mlp.backward(params, np.array([[x]]), np.array([[t]]))
    for gg, e in zip(grads, expect):
        assert abs(float(gg.reshape(-1)[0]) - e) < 1e-14


def test_bf16_rounding_values():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 3.0e-3])
    r = mlp.round_bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # tie rounds to even
    assert r[2] == 1.0 + 2.0 ** -7        # rounds up
    assert r[3] == -2.5
    assert abs(r[4] - 3.0e-3) < 2 ** -8 * 3.0e-3


def test_adam_first_step_is_signed_lr():
    params = [np.array([1.0, -2.0, 0.5])]
    grads = [np.array([0.3, -4.0, 1e-3])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    params, m, v = mlp.adam_step(params, grads, m, v, 1, lr=0.01)
    assert np.allclose(params[0], np.array([1.0, -2.0, 0.5]) - 0.01 * np.sign(grads[0]), atol=1e-7)


def test_training_reduces_loss():
    g = np.random.default_rng(0)
    params = W.mlp_init(4, 16, 2, 1)
    X = g.standard_normal((64, 4))
    T = np.stack([X[:, 0] - X[:, 1], np.maximum(X[:, 2], 0)], axis=1)
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    l0 = mlp.loss(params, X, T)
    for t in range(1, 201):
        gr = mlp.backward(params, X, T)
        params, m, v = mlp.adam_step(params, gr, m, v, t, lr=1e-2)
    assert mlp.loss(params, X, T) < 0.2 * l0
