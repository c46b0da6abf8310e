"""FP64 reference of the error-bar surrogate network (test infrastructure only).

The surrogate is not in the paper (Section 4 estimates error bars by brute
Monte Carlo over 250 realisations); this reference defines what the CUDA
kernels must compute so their gradients can be checked:

    xn = (x - mu_x) / sd_x                      (per feature)
    h1 = tanh(W1 xn + b1),  h2 = tanh(W2 h1 + b2)
    yn = w3 . h2 + b3,      y = yn * sd_y + mu_y
    loss = mean over rows of (yn - (t - mu_y)/sd_y)^2

W1, W2, w3 enter as BF16 values (the matmul operands of the kernels); biases
are FP32.  Gradients are w.r.t. (W1, b1, W2, b2, w3, b3), by the chain rule
written out layer by layer; pinned by central finite differences in
tests/test_oracle_mlp.py.  Flat parameter order:
    W1 [w, d] | b1 [w] | W2 [w, w] | b2 [w] | w3 [w] | b3 [1]
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(p, d, w):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + w * d].reshape(w, d); o += w * d
    b1 = p[o:o + w]; o += w
    W2 = p[o:o + w * w].reshape(w, w); o += w * w
    b2 = p[o:o + w]; o += w
    w3 = p[o:o + w]; o += w
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def n_params(d, w):
    return w * d + w + w * w + w + w + 1


def forward(p, x, d, w, norm, bf16=True):
    """Returns (y, cache).  norm = (mu_x [d], sd_x [d], mu_y, sd_y)."""
    W1, b1, W2, b2, w3, b3 = unflatten(p, d, w)
    if bf16:
        W1, W2, w3 = bf16_round(W1), bf16_round(W2), bf16_round(w3)
    mu_x, sd_x, mu_y, sd_y = norm
    xn = (np.asarray(x, dtype=np.float64) - mu_x) / sd_x
    h1 = np.tanh(xn @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    yn = h2 @ w3 + b3
    return yn * sd_y + mu_y, (xn, h1, h2, yn, W1, W2, w3)


def loss_and_grad(p, x, t, d, w, norm, bf16=True):
    """Mean squared error on the normalised target and its gradient (flat)."""
    y, (xn, h1, h2, yn, W1, W2, w3) = forward(p, x, d, w, norm, bf16)
    mu_y, sd_y = norm[2], norm[3]
    tn = (np.asarray(t, dtype=np.float64) - mu_y) / sd_y
    n = xn.shape[0]
    r = yn - tn
    loss = np.mean(r * r)
    dyn = 2.0 * r / n                      # dL/dyn
    g_w3 = h2.T @ dyn
    g_b3 = dyn.sum()
    dz2 = np.outer(dyn, w3) * (1.0 - h2 * h2)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    g_W1 = dz1.T @ xn
    g_b1 = dz1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g
