"""Exact model of the FP64 path's FP32 overload screen (Eqs. rank_correct, sfr_pen-zctg), and a grid
built to defeat a screen whose margin does not follow its error bound.

The FP64 path screens every post-contingency element F = f_m + L f_k in FP32 and recomputes the
candidates in FP64; an element is overloaded when F^2 + qmax2 - s_ctg^2 > 0 in FP64.  For that
classification to be FP64's, the screen may never reject an element that FP64 counts as overloaded.
This module replays the screen's single-precision operations exactly (each one rounded to nearest
from the exact rational result), so the tests can check that property on chosen inputs.

Only tests import this module.
"""
from fractions import Fraction as Fr

import numpy as np

import oracle
import synth
from oracle import qg_oracle as Q


def rn32(q):
    """The float32 nearest to the rational q (ties to even)."""
    f = np.float32(float(q))  # within one float32 step of the answer
    best = f
    for c in (np.nextafter(f, np.float32(-np.inf)), np.nextafter(f, np.float32(np.inf))):
        dc, db = abs(Fr(float(c)) - q), abs(Fr(float(best)) - q)
        if dc < db or (dc == db and int(np.array(c).view(np.int32)) % 2 == 0):
            best = c
    return best


def fma32(a, b, c):
    return rn32(Fr(float(a)) * Fr(float(b)) + Fr(float(c)))


def add32(a, b):
    return rn32(Fr(float(a)) + Fr(float(b)))


def mul32(a, b):
    return rn32(Fr(float(a)) * Fr(float(b)))


def fma64(a, b, c):
    return float(Fr(a) * Fr(b) + Fr(c))  # float(Fraction) rounds to nearest


def exact_overload(fm, L, fk, q2, s2):
    """The FP64 path's decision on a candidate: fma(Fx, Fx, q2) - s2 > 0 with Fx = fma(L, f_k, f_m)."""
    Fx = fma64(L, fk, fm)
    return fma64(Fx, Fx, q2) - s2 > 0.0


def screen_margin(fm, L, fk, q2, s2):
    """The screen with the margin derived from the FP32 error bound (one column: the thread's row and
    column maxima are this element's own magnitudes, the tightest case).  True: a candidate."""
    qs = np.float32((q2 - s2) + 2.0 ** -22 * (abs(q2 - s2) + s2))
    L32, fk32, fm32 = np.float32(L), np.float32(fk), np.float32(fm)
    ah = fma32(abs(L32), abs(fk32), abs(fm32))
    qs = add32(qs, mul32(mul32(ah, ah), np.float32(2.0 ** -21)))
    F = fma32(L32, fk32, fm32)
    return fma32(F, F, qs) >= 0


def screen_fixed(fm, L, fk, q2, s2, rel=1e-4):
    """A screen with a fixed margin rel * s_ctg^2 (not tied to |f_m| + |L||f_k|).  True: a candidate."""
    qs = add32(np.float32(q2 - s2), mul32(np.float32(rel), np.float32(s2)))
    F = fma32(np.float32(L), np.float32(fk), np.float32(fm))
    return fma32(F, F, qs) > 0


# ------------------------------------------------------------------------------------------------
# a grid where a large loop flow cancels under an outage
# ------------------------------------------------------------------------------------------------

RING_X = 1e-5 * np.array([1.0, 1.37, 0.83, 1.19])  # series reactances (lossless, no charging)
LOAD = 0.4731
MON = 2        # the monitored branch (bus 2 -> bus 3)


def ring_case(phi, s_ctg_mon=1e6):
    """Four buses in a ring, branches 0: 0->1, 1: 1->2, 2: 2->3, 3: 3->0; branch 3 is a phase shifter.
    Its shift drives a loop flow of phi / sum(x) (about 6,900 pu at phi = 0.3) around the ring, on
    top of the 0.47 pu that the generator at bus 0 sends to the load at bus 2.  An outage of branch 0
    or 1 opens the loop: the monitored branch 2 then carries the 0.47 pu alone, so its
    post-contingency flow is f_2 + L f_k with |f_2|, |L f_k| near 6,900 and their sum near 0.47.
    Balance prices are 1 (the AC flow on branch 0 is large at the point used)."""
    one = np.ones(1)
    M = 4
    return synth.Case(
        name="ring4", seed=0, n_bus=4, n_branch=M, n_gen=1, n_zone=1, ref_bus=0,
        br_from=np.array([0, 1, 2, 3], np.int32), br_to=np.array([1, 2, 3, 0], np.int32),
        br_r=np.zeros(M), br_x=RING_X.copy(), br_b=np.zeros(M), s_max=np.full(M, 1e6),
        s_max_ctg=np.array([1e6, 1e6, s_ctg_mon, 1e6]), gen_bus=np.array([0], np.int32),
        gen_zone=np.array([0], np.int32), cost_a=0.05 * one, cost_b=20.0 * one, cost_r=2.0 * one,
        pmin=0 * one, pmax=2.0 * one, qmin=-one, qmax=one, ramp=one, vmin=np.full(4, 0.9),
        vmax=np.full(4, 1.1), T=1, dt=one, load_p=np.array([[0.0, 0.0, LOAD, 0.0]]),
        load_q=np.zeros((1, 4)), reserve_req=np.zeros((1, 1)), bus_zone=np.zeros(4, np.int32),
        ctg=np.array([0, 1, 2], np.int32), xf_branch=np.array([3], np.int32), tau_min=np.array([0.9]),
        tau_max=np.array([1.1]), phi_min=np.array([-0.5]), phi_max=np.array([0.5]), c_p=1.0, c_q=1.0)


def ring_point(case, phi):
    """v = 1; theta = (0, phi, phi, phi) so that only branch 0 carries AC flow (the monitored branch's
    q is 0 and its s is |F|); p = the load at the one generator, q = r = 0; tau = 1, phi."""
    th = np.array([[0.0, phi, phi, phi]])
    return oracle.pack(np.ones((1, 4)), th, np.array([[LOAD]]), np.zeros((1, 1)), np.zeros((1, 1)),
                       np.ones((1, 1)), np.full((1, 1), phi))


def ring_elements(case, x):
    """FP64 base flows f (M,) with the phase shifter's own flow, and the line-outage block L (M, K):
    L[m, k] = y_m a_m^T Yhat^-1 a_k / (1 - y_k a_k^T Yhat^-1 a_k), 0 on the outaged branch itself."""
    _, _, p, _, _, tau, phi = oracle.unpack(case, x)
    net = oracle.dc_network(case)
    _, pbar = oracle.dc_injections(case, p)
    bflow = Q.phase_shift_flows(case, net, Q.branch_tau_phi(case, tau, phi)[1])
    _, f = oracle.dc_base_flows(case, net, pbar, bflow)
    U, den = Q.outage_columns(case, net)
    Eh = net.E[:, net.keep]
    L = (net.y[:, None] * (Eh @ U)) / den[None, :]
    L[case.ctg, np.arange(case.K)] = 0.0
    return f[0], L


def dropped_by_fixed_margin():
    """A ring case, a point and an outage k whose element (MON, k) FP64 counts as overloaded but the
    fixed-margin screen rejects: the rating s_ctg of branch MON is set just under |F| by half the
    gap the FP32 rounding opens.  Returns (case, x, k, details)."""
    for phi in np.linspace(0.30, 0.20, 41):
        c0 = ring_case(phi)
        x = ring_point(c0, phi)
        f, L = ring_elements(c0, x)
        for kk, k in enumerate(c0.ctg):
            if k == MON:
                continue
            fm, fk, Lmk = f[MON], f[k], L[MON, kk]
            F64 = fma64(Lmk, fk, fm)
            F32 = float(fma32(np.float32(Lmk), np.float32(fk), np.float32(fm)))
            D = abs(F64) - abs(F32)  # the FP32 value's shortfall in magnitude
            if D <= 1e-4 * abs(F64):
                continue
            s2 = F64 * F64 - abs(F64) * D
            if not (exact_overload(fm, Lmk, fk, 0.0, s2) and not screen_fixed(fm, Lmk, fk, 0.0, s2)):
                continue
            c = ring_case(phi, np.sqrt(s2))
            return c, x, kk, dict(phi=phi, fm=fm, fk=fk, L=Lmk, F64=F64, F32=F32, s2=s2)
    raise AssertionError("no ring configuration defeats the fixed margin")
