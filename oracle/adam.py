"""FP64 projected Adam (Alg. 3) and the wall-clock schedules of Sec. II-F.

TEST INFRASTRUCTURE ONLY (see qg_oracle.py).
"""
from __future__ import annotations

import math

import numpy as np


def adam_step(x, m, v, g, i, lr, beta1, beta2, eps, lo, hi, paper_eps=False):
    """One step of Alg. 3 for every basis variable (period loop fused), then the clip of Alg. 3.

    Default form is the textbook Adam step  x -= lr * mhat / (sqrt(vhat) + eps)  (Kingma & Ba).
    paper_eps=True takes the numerator literally as printed in Alg. 3, (mhat + eps).
    i is the 1-based step count used in the bias corrections.
    Returns new (x, m, v); inputs are not modified.
    """
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** i)
    vhat = v / (1.0 - beta2 ** i)
    num = mhat + eps if paper_eps else mhat
    x = x - lr * num / (np.sqrt(vhat) + eps)
    x = np.minimum(np.maximum(x, lo), hi)
    return x, m, v


def normalized_time(tw, t0, tf):
    """Eq. norm_t: map [t0, tf] onto [-1, 1]."""
    return 2.0 * (tw - t0) / (tf - t0) - 1.0


def magnitude_scale(that):
    """Eq. mag_scale: reflected sigmoid e^{4 t} / (0.6 + e^{4 t})."""
    e = math.exp(4.0 * that)
    return e / (0.6 + e)


def step_size(alpha0, alphaf, tw, t0, tf):
    """Eq. step_size: alpha0 * 10^(beta * log10(alphaf / alpha0))."""
    b = magnitude_scale(normalized_time(tw, t0, tf))
    return alpha0 * 10.0 ** (b * math.log10(alphaf / alpha0))


def schedule_table(iters, lr0, lrf, eps0, epsf, beta0, beta1, lag):
    """Per-iteration (lr, eps, beta) of Sec. II-F with time measured as the iteration fraction:
    lr from Eqs. norm_t, mag_scale, step_size over [0, iters - 1]; eps with the same law over its
    own range, its normalized time lagging by `lag` (the step size decay leads the tightening);
    beta rising linearly from beta0 to beta1 (the homotopy scale)."""
    out = np.zeros((iters, 3))
    for i in range(iters):
        if iters > 1:
            that = normalized_time(i, 0, iters - 1)
        else:
            that = -1.0
        out[i, 0] = step_size(lr0, lrf, i, 0, max(iters - 1, 1)) if iters > 1 else \
            lr0 * 10.0 ** (magnitude_scale(-1.0) * math.log10(lrf / lr0))
        out[i, 1] = eps0 * 10.0 ** (magnitude_scale(that - lag) * math.log10(epsf / eps0))
        out[i, 2] = beta0 + (beta1 - beta0) * (that + 1.0) / 2.0
    return out
