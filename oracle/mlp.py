"""Oracle: the parameter model's MLP in FP64 numpy (test infrastructure only).

n_in -> h (tanh) -> h (tanh) -> n_out, packed parameters
[W1 (h x n_in), b1, W2 (h x h), b2, W3 (n_out x h), b3]; loss = mean over all
batch x n_out entries of the squared error of standardised outputs, with
inputs standardised as (x - in_mean)/in_std and targets as
(y - out_mean)/out_std.  Backpropagation written out layer by layer.
Pinned by central finite differences (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np


def unpack(p, n_in, h, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in ((h, n_in), (h,), (h, h), (h,), (n_out, h), (n_out,)):
        size = int(np.prod(shape))
        out.append(p[o:o + size].reshape(shape))
        o += size
    return out


def forward(p, X, n_in, h, n_out, norm=None):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h, n_out)
    X = np.asarray(X, dtype=np.float64)
    if norm is not None:
        X = (X - norm[0]) / norm[1]
    A1 = np.tanh(X @ W1.T + b1)
    A2 = np.tanh(A1 @ W2.T + b2)
    Z3 = A2 @ W3.T + b3
    if norm is not None:
        return norm[2] + norm[3] * Z3
    return Z3


def loss_grad(p, X, Y, n_in, h, n_out, norm=None):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h, n_out)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if norm is not None:
        X = (X - norm[0]) / norm[1]
        Y = (Y - norm[2]) / norm[3]
    A1 = np.tanh(X @ W1.T + b1)
    A2 = np.tanh(A1 @ W2.T + b2)
    Z3 = A2 @ W3.T + b3
    R = Z3 - Y
    cnt = R.size
    loss = float((R * R).sum() / cnt)
    dZ3 = 2.0 * R / cnt
    gW3 = dZ3.T @ A2
    gb3 = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ W3) * (1.0 - A2 * A2)
    gW2 = dZ2.T @ A1
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * (1.0 - A1 * A1)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
