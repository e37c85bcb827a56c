"""Exact model of the contingency screen's bound test (Sec. II-E screen; the argument is at the kernel).

A warp skips a chunk when Lmax fc < r for each of its rows, with r the row's clearance
rd(rd(sqrt_rd(s_ctg^2 - qmax2)) (1 - 2^-20)) - |f_m|) (every step rounded down; -1 below 2^-40).  The
claim is that then no element of the chunk is a candidate of the FP32 screen: not on the mixed path
(fma(F, F, qs) > 0) and not on the FP64 path (its margin added, fma(F, F, qs') >= 0).  These tests
replay the kernel's single-precision operations exactly (rational arithmetic, then the rounding the
kernel's instruction uses) on the worst element of a cleared piece (|L| = Lmax, |f_k| = fc, L f_k of
f_m's sign), with Lmax fc pushed right up to the bound; and check that the construction is not
vacuous: past the true clearance the same element is a candidate.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from screen_model import add32, fma32, mul32, rn32

ONE_MINUS = Fr(1) - Fr(1, 2 ** 20)
FLOOR = Fr(1, 2 ** 40)


def f32(x):
    return np.float32(x)


def rd32(q):
    """The largest float32 not above the rational q."""
    f = rn32(q)
    if Fr(float(f)) > q:
        f = np.nextafter(f, np.float32(-np.inf))
    return f


def sqrt_rd32(a):
    """The largest float32 s >= 0 with s^2 <= a (a a non-negative float32)."""
    A = Fr(float(a))
    s = np.float32(np.sqrt(np.float64(a)))
    while Fr(float(s)) ** 2 > A:
        s = np.nextafter(s, np.float32(-np.inf))
    while Fr(float(np.nextafter(s, np.float32(np.inf)))) ** 2 <= A:
        s = np.nextafter(s, np.float32(np.inf))
    return s


def clear_margin(fm, qs, factor=ONE_MINUS):
    """The kernel's clear_margin: float32 r, or -1 where the margin is below 2^-40 or undefined."""
    if not (-float(qs) >= 0.0) or not np.isfinite(fm):  # an infinite flow: r = -inf in the kernel
        return f32(-1.0)
    s = sqrt_rd32(f32(-float(qs)))
    m = rd32(Fr(float(s)) * factor)
    r = rd32(Fr(float(m)) - abs(Fr(float(fm))))
    return r if Fr(float(r)) >= FLOOR else f32(-1.0)


def bound_clear(lmax, fc, r):
    """fma(-Lmax, fc, r) > 0 rounded to nearest (what the kernel's paired FMA and compare decide)."""
    return float(rn32(Fr(float(r)) - Fr(float(lmax)) * Fr(float(fc)))) > 0.0


def screen_mixed(L, fk, fm, qs):
    F = fma32(L, fk, fm)
    return float(fma32(F, F, qs)) > 0.0


def screen_fp64(L, fk, fm, qs, lrow, fkq):
    ah = fma32(lrow, fkq, abs(fm))
    qs2 = add32(qs, mul32(mul32(ah, ah), f32(2.0 ** -21)))
    F = fma32(L, fk, fm)
    return float(fma32(F, F, qs2)) >= 0.0


def qs_mixed(q2, s2):
    return add32(q2, -s2)  # (float)(q2 - s2) with float operands


def qs_fp64(q2, s2):
    return np.float32((q2 - s2) + 2.0 ** -22 * (abs(q2 - s2) + s2))


def worst_element(fm, lmax, fc):
    """The element of largest |F| a cleared piece can hold: |L| = Lmax, |f_k| = fc, L f_k of f_m's sign."""
    sg = f32(-1.0) if fm < 0 else f32(1.0)
    return f32(sg * lmax), fc


def cases(rng, n):
    """Rows (f_m, q2, s2) over many magnitudes, with the rating above the reactive flow."""
    out = []
    for _ in range(n):
        scale = 10.0 ** rng.uniform(-6, 6)
        s2 = (scale * rng.uniform(0.5, 2.0)) ** 2
        q2 = s2 * rng.uniform(0.0, 0.999) ** 2
        fm = scale * rng.uniform(-1.5, 1.5)
        out.append((fm, q2, s2))
    return out


def split(r, rng):
    """Lmax, fc (float32, positive) with Lmax fc as close below r as float32 allows."""
    fc = f32(float(r) * 10.0 ** rng.uniform(-3, 3))
    lmax = rd32(Fr(float(r)) / Fr(float(fc)))
    while not Fr(float(lmax)) * Fr(float(fc)) < Fr(float(r)):
        lmax = np.nextafter(lmax, np.float32(-np.inf))
    return lmax, fc


def cleared_candidates(path, n, seed, factor=ONE_MINUS):
    """(pieces the bound test clears, candidates among their worst elements) over n rows."""
    rng = np.random.default_rng(seed)
    cleared = bad = 0
    for fm, q2, s2 in cases(rng, n):
        qs = qs_mixed(f32(q2), f32(s2)) if path == "mixed" else qs_fp64(q2, s2)
        fm32 = f32(fm)
        r = clear_margin(fm32, qs, factor)
        if float(r) < 0:
            continue
        lmax, fc = split(r, rng)
        if not bound_clear(lmax, fc, r):
            continue
        cleared += 1
        L, fk = worst_element(fm32, lmax, fc)
        bad += screen_mixed(L, fk, fm32, qs) if path == "mixed" else screen_fp64(L, fk, fm32, qs, lmax, fc)
    return cleared, bad


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_a_cleared_piece_has_no_candidate(path):
    cleared, bad = cleared_candidates(path, 1500, 11 if path == "mixed" else 12)
    assert cleared > 500 and bad == 0, (cleared, bad)


def test_the_margin_factor_is_needed_on_the_fp64_path():
    """With the clearance taken as sqrt_rd(s_ctg^2 - qmax2) - |f_m| (no factor 1 - 2^-20), the FP64
    path's screen margin makes nearly every cleared worst element a candidate: the factor is what
    covers that margin."""
    cleared, bad = cleared_candidates("fp64", 400, 12, factor=Fr(1))
    assert cleared > 200 and bad > 0.9 * cleared, (cleared, bad)


def test_past_the_clearance_the_worst_element_is_a_candidate():
    """The construction is not vacuous: with Lmax fc 2^-10 above the exact clearance
    sqrt(s2 - q2) - |f_m| the same element is a candidate of the mixed screen."""
    rng = np.random.default_rng(13)
    flagged = total = 0
    for fm, q2, s2 in cases(rng, 800):
        q2f, s2f, fm32 = f32(q2), f32(s2), f32(fm)
        qs = qs_mixed(q2f, s2f)
        if not float(qs) < 0:
            continue
        c = np.sqrt(-np.float64(qs)) - abs(np.float64(fm32))
        if c <= 0:
            continue
        total += 1
        target = c * (1 + 2.0 ** -10)
        fc = f32(target * 10.0 ** rng.uniform(-2, 2))
        lmax = f32(target / np.float64(fc))
        L, fk = worst_element(fm32, lmax, fc)
        flagged += screen_mixed(L, fk, fm32, qs)
    assert total > 300 and flagged >= 0.99 * total, (flagged, total)


def test_margin_edge_cases():
    # no clearance where the reactive flow alone reaches the rating, or where inputs are not finite
    assert float(clear_margin(f32(0.0), f32(0.0))) == -1.0
    assert float(clear_margin(f32(0.0), f32(1.0))) == -1.0
    assert float(clear_margin(f32(np.nan), f32(-1.0))) == -1.0
    assert float(clear_margin(f32(np.inf), f32(-1.0))) == -1.0
    # below the 2^-40 floor: no clearance
    assert float(clear_margin(f32(0.0), f32(-(2.0 ** -82)))) == -1.0
    # a clear row: r is below sqrt(-qs) (1 - 2^-20) - |f_m| and within a few ulps of it
    r = clear_margin(f32(0.25), f32(-1.0))
    assert 0 < float(r) <= (1 - 2.0 ** -20) - 0.25 and float(r) > 0.75 - 2.0 ** -18
