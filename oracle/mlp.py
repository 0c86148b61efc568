"""Two-hidden-layer ReLU MLP used for the learned ADMM warm start: forward
pass, backward pass of the mean-squared error and one Adam step, in FP64.

Test infrastructure only (see oracle/__init__.py).  The paper has no learned
component; this is the plain definition of the network the CUDA kernels train.

Network:  h1 = relu(X W1^T + b1),  h2 = relu(h1 W2^T + b2),  Y = h2 W3^T + b3
Loss:     L = (1 / (2 B)) * sum over batch and outputs of (Y - T)^2
Adam:     m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
          w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

round_bf16 mimics storing an operand in bfloat16 (round to nearest even) so
that the oracle can take the same rounding decisions as a kernel that feeds
BF16 operands to the tensor cores.
"""
from __future__ import annotations

import numpy as np


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, X, bf16: bool = False):
    W1, b1, W2, b2, W3, b3 = params
    r = round_bf16 if bf16 else (lambda a: a)
    z1 = r(X) @ r(W1).T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = r(h1) @ r(W2).T + b2
    h2 = np.maximum(z2, 0.0)
    Y = r(h2) @ r(W3).T + b3
    return Y, (X, z1, h1, z2, h2)


def loss(params, X, T, bf16: bool = False) -> float:
    Y, _ = forward(params, X, bf16)
    return float(0.5 * np.sum((Y - T) ** 2) / X.shape[0])


def backward(params, X, T, bf16: bool = False):
    """Gradients of loss() w.r.t. (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    r = round_bf16 if bf16 else (lambda a: a)
    Y, (X, z1, h1, z2, h2) = forward(params, X, bf16)
    Bn = X.shape[0]
    dY = (Y - T) / Bn
    gW3 = r(dY).T @ r(h2)
    gb3 = dY.sum(axis=0)
    dh2 = r(dY) @ r(W3)
    dz2 = dh2 * (z2 > 0)
    gW2 = r(dz2).T @ r(h1)
    gb2 = dz2.sum(axis=0)
    dh1 = r(dz2) @ r(W2)
    dz1 = dh1 * (z1 > 0)
    gW1 = r(dz1).T @ r(X)
    gb1 = dz1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; t counts steps from 1."""
    for i in range(len(params)):
        m[i] = beta1 * m[i] + (1 - beta1) * grads[i]
        v[i] = beta2 * v[i] + (1 - beta2) * grads[i] ** 2
        mh = m[i] / (1 - beta1 ** t)
        vh = v[i] / (1 - beta2 ** t)
        params[i] = params[i] - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v
