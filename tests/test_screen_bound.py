"""The FP64 path's overload screen keeps every element that FP64 counts as overloaded.

The screen evaluates F = f_m + L f_k and F^2 + qmax2 - s_ctg^2 in FP32 with a margin; candidates
are recomputed in FP64.  Its margin follows from an error bound (u = 2^-24): the FP32 value of F is
within 3.0001 u (|f_m| + |L||f_k|) of F, so F^2 moves by at most 6.0003 u A^2 (A = |f_m| + |L||f_k|),
and q2 - s2 by u |q2 - s2| when rounded; the screen adds 2^-21 Ahat^2 + 2^-22 (|q2 - s2| + s2) with
Ahat >= A computed from the FP32 inputs, and keeps elements whose sum is >= 0.  These tests replay
the screen's FP32 operations exactly (tests/screen_model.py) at inputs built to sit on the edge."""
import numpy as np

from screen_model import (MON, dropped_by_fixed_margin, exact_overload, screen_fixed, screen_margin)


def _edge_inputs(rng, n):
    """Elements with heavy cancellation (|f_m|, |L f_k| up to ~1e4 times |F|) whose FP64 value sits
    just above or just below the limit."""
    out = []
    for _ in range(n):
        fk = rng.uniform(-1000, 1000)
        L = rng.uniform(-2, 2)
        fm = -L * fk + rng.uniform(-0.5, 0.5)
        q2 = 0.0 if rng.random() < 0.5 else rng.uniform(0, 1)
        F = fm + L * fk
        gap = 2 * abs(F) * (abs(fm) + abs(L * fk)) * 2.0 ** -24 * rng.uniform(-4, 4)  # ~ the FP32 error of F^2
        s2 = max(F * F + q2 - gap, 1e-6)
        out.append((fm, L, fk, q2, s2))
    return out


def test_margin_never_drops_an_fp64_overload():
    rng = np.random.default_rng(0)
    n_over = n_fixed_miss = 0
    for fm, L, fk, q2, s2 in _edge_inputs(rng, 3000):
        if exact_overload(fm, L, fk, q2, s2):
            n_over += 1
            assert screen_margin(fm, L, fk, q2, s2), (fm, L, fk, q2, s2)
            n_fixed_miss += not screen_fixed(fm, L, fk, q2, s2)
    assert n_over > 1000
    assert n_fixed_miss >= 5  # a margin of 1e-4 s_ctg^2 misses some of them


def test_margin_keeps_the_screen_selective():
    """Away from the limit (|F^2 + q2 - s2| above the bound) the screen still rejects."""
    rng = np.random.default_rng(1)
    rejected = 0
    for fm, L, fk, q2, s2 in _edge_inputs(rng, 500):
        A = abs(fm) + abs(L * fk)
        s2_far = (fm + L * fk) ** 2 + q2 + 64 * 2.0 ** -24 * (A * A + s2)  # clearly not overloaded
        rejected += not screen_margin(fm, L, fk, q2, s2_far)
    assert rejected == 500


def test_ring_element_defeats_a_fixed_margin():
    """On the phase-shifter ring the element (monitored branch, outage) is overloaded in FP64, the
    fixed-margin screen rejects it, and the derived margin keeps it."""
    c, x, kk, e = dropped_by_fixed_margin()
    assert abs(e["fm"]) > 5000 and abs(e["F64"]) < 1.0  # a cancellation of ~10,000 to 1
    assert exact_overload(e["fm"], e["L"], e["fk"], 0.0, e["s2"])
    assert not screen_fixed(e["fm"], e["L"], e["fk"], 0.0, e["s2"])
    assert screen_margin(e["fm"], e["L"], e["fk"], 0.0, e["s2"])
    assert c.s_max_ctg[MON] ** 2 < e["F64"] ** 2
