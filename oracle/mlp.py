"""Multilayer perceptron 4 -> 64 -> 64 -> O with tanh hidden layers, FP64
(test infrastructure: only tests/ may use it).

This is the plain definition of the network whose training kernels the GPU
library implements for the learned preconditioner sums: forward pass,
mean-squared-error loss over the batch and the outputs, and the gradient
written out by the chain rule (no automatic differentiation). The parameter
vector follows the library's layout: W1 (64 x 4, one row per output unit),
b1 (64), W2 (64 x 64), b2 (64), W3 (O x 64), b3 (O). The gradient is pinned
by central finite differences in tests/test_mlp_oracle.py.
"""
from __future__ import annotations

import numpy as np

H, IN = 64, 4


def n_params(O: int) -> int:
    return H * IN + H + H * H + H + O * H + O


def unpack(p, O):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    out = []
    for shape in ((H, IN), (H,), (H, H), (H,), (O, H), (O,)):
        size = int(np.prod(shape))
        out.append(p[i:i + size].reshape(shape))
        i += size
    return out


def forward(p, X, O):
    """Y (B x O) and the hidden activations."""
    W1, b1, W2, b2, W3, b3 = unpack(p, O)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, (X, h1, h2)


def loss_and_grad(p, X, T, O):
    """MSE = mean over batch and outputs of (Y - T)^2, and its gradient (flat)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, O)
    Y, (X, h1, h2) = forward(p, X, O)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    d = Y - T
    loss = float(np.sum(d * d) / (B * O))
    dY = 2.0 * d / (B * O)
    gW3 = dY.T @ h2
    gb3 = dY.sum(0)
    d2 = (dY @ W3) * (1.0 - h2 * h2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad


def loss_only(p, X, T, O):
    Y, _ = forward(p, X, O)
    d = Y - np.asarray(T, dtype=np.float64)
    return float(np.sum(d * d) / d.size)
