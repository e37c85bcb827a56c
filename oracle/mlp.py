"""FP64 oracle of the warm-start MLP's forward and backward pass.

TEST INFRASTRUCTURE ONLY (see qg_oracle.py).

Network:  Z1 = X W1^T + b1, H1 = relu(Z1), Z2 = H1 W2^T + b2, H2 = relu(Z2), Y = H2 W3^T + b3,
loss = mean((Y - target)^2).  With ``quantize=True`` every GEMM operand is rounded to BF16 at the
points where the GPU rounds it (X, H1, H2, the weights, dY, dZ2, dZ1), with straight-through
gradients; everything else is FP64.  With ``quantize=False`` it is the plain FP64 network, whose
gradient is pinned by finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def split(params, n_in, n_h, n_out):
    o = 0
    W1 = params[o:o + n_h * n_in].reshape(n_h, n_in); o += n_h * n_in
    b1 = params[o:o + n_h]; o += n_h
    W2 = params[o:o + n_h * n_h].reshape(n_h, n_h); o += n_h * n_h
    b2 = params[o:o + n_h]; o += n_h
    W3 = params[o:o + n_out * n_h].reshape(n_out, n_h); o += n_out * n_h
    b3 = params[o:o + n_out]
    return W1, b1, W2, b2, W3, b3


def forward_backward(params, X, target, n_in, n_h, n_out, quantize=True):
    """Returns (Y, loss, grad) with grad in the parameter layout W1, b1, W2, b2, W3, b3."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    params = np.asarray(params, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = split(params, n_in, n_h, n_out)
    Xq, W1q, W2q, W3q = q(X), q(W1), q(W2), q(W3)
    Z1 = Xq @ W1q.T + b1
    H1q = q(np.maximum(Z1, 0.0))
    Z2 = H1q @ W2q.T + b2
    H2q = q(np.maximum(Z2, 0.0))
    Y = H2q @ W3q.T + b3
    R = Y - target
    loss = float(np.mean(R * R))
    dY = 2.0 * R / R.size
    dYq = q(dY)
    gW3 = dYq.T @ H2q
    gb3 = dY.sum(axis=0)
    dZ2 = (dYq @ W3q) * (Z2 > 0)
    dZ2q = q(dZ2)
    gW2 = dZ2q.T @ H1q
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2q @ W2q) * (Z1 > 0)
    dZ1q = q(dZ1)
    gW1 = dZ1q.T @ Xq
    gb1 = dZ1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return Y, loss, grad


def loss_only(params, X, target, n_in, n_h, n_out):
    return forward_backward(params, X, target, n_in, n_h, n_out, quantize=False)[1]
