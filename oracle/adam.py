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
