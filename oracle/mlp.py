"""FP64 reference of the warm-start perceptron -- TEST INFRASTRUCTURE (see ``oracle/__init__``).

Plain NumPy forward and backward of the three-layer perceptron x -> tanh(W1 x + b1) ->
tanh(W2 a1 + b2) -> W3 a2 + b3 with the mean-squared-error loss mean((y - t)^2), written from the
definitions (chain rule, layer by layer).  Parameters are flat in the order W1 [H][I], b1, W2 [H][H],
b2, W3 [O][H], b3.  ``bf16`` rounds the weight matrices to bfloat16 (round to nearest even) the way
the GPU's working copy is made, so that the GPU gradients can be compared with a reference that
sees the same weights.
"""
from __future__ import annotations

import numpy as np


def split(params: np.ndarray, n_in: int, H: int, n_out: int):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * n_in].reshape(H, n_in); o += H * n_in
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + n_out * H].reshape(n_out, H); o += n_out * H
    b3 = p[o:o + n_out]; o += n_out
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even) and return them as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, n_in, H, n_out, bf16=False):
    W1, b1, W2, b2, W3, b3 = split(params, n_in, H, n_out)
    if bf16:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    x = np.asarray(x, dtype=np.float64)
    a1 = np.tanh(x @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    y = a2 @ W3.T + b3
    return y, (x, a1, a2, W1, W2, W3)


def loss_and_grad(params, x, t, n_in, H, n_out, bf16=False):
    y, (x, a1, a2, W1, W2, W3) = forward(params, x, n_in, H, n_out, bf16)
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / n                  # d loss / d y
    gW3 = dy.T @ a2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * (1.0 - a2 ** 2)       # through tanh
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - a1 ** 2)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
