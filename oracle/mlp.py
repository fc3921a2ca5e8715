"""Plain FP64 forward/backward of the learned guess's networks (numpy).

TEST INFRASTRUCTURE ONLY: checks the gradients the CUDA training kernels
compute.  Shares no code with the library.

Network: y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 with 64 hidden units per
layer, scalar input x, k outputs; loss = mean over samples and outputs of
(y - target)^2.  Parameters are a flat vector in the layout
W1[64], b1[64], W2[64][64] (row = output unit), b2[64], W3[k][64], b3[k].
"""
from __future__ import annotations

import numpy as np

H = 64


def unpack(p, k):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H]; o += H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + k * H].reshape(k, H); o += k * H
    b3 = p[o:o + k]; o += k
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def n_params(k):
    return 3 * H + H * H + k * H + k


def forward(p, k, x):
    """x: (n,) -> y: (k, n)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, k)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(np.outer(W1, x) + b1[:, None])
    h2 = np.tanh(W2 @ h1 + b2[:, None])
    return W3 @ h2 + b3[:, None]


def loss_and_grad(p, k, x, y):
    """Mean squared error over the k x n outputs and its gradient (flat)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, k)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(k, -1)
    n = x.size
    h1 = np.tanh(np.outer(W1, x) + b1[:, None])
    h2 = np.tanh(W2 @ h1 + b2[:, None])
    out = W3 @ h2 + b3[:, None]
    err = out - y
    loss = float(np.sum(err ** 2) / (k * n))
    dout = 2.0 * err / (k * n)
    gW3 = dout @ h2.T
    gb3 = dout.sum(axis=1)
    dz2 = (W3.T @ dout) * (1.0 - h2 ** 2)
    gW2 = dz2 @ h1.T
    gb2 = dz2.sum(axis=1)
    dz1 = (W2.T @ dz2) * (1.0 - h1 ** 2)
    gW1 = dz1 @ x
    gb1 = dz1.sum(axis=1)
    g = np.concatenate([gW1, gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
