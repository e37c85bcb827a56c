"""Value pins of every penalty family of the FP64 oracle.

The finite-difference pins fix each gradient against its own objective; these fix the objective
values themselves.  A hand-built two-bus, two-period case with two devices in two reserve zones puts
each family in a state where its value can be written out directly from the paper's definitions,
with scalar arithmetic and complex numbers (no numpy broadcasting, no code shared with the oracle):

* energy cost and reserve cost, sum_t d_t sum_g (a p^2 + b p + c_r r)          (Eq. nlp_updated)
* balance, sum_t d_t c beta |P_it|_s, |x|_s = sqrt(x^2 + eps^2)                 (Example 4)
* thermal, sum_t d_t c_s beta sigma_s(max(|S_fr|, |S_to|) - s_max)            (Example 1)
* zonal reserve shortfall, sum_t d_t c_rz beta sigma_s(R_zt - sum_{g in z} r_gt)
* headroom rho beta sigma_s(p + r - Pmax) and ramps rho beta sigma_s(+-(p_t - p_{t-1}) - R d_t)
  (the penalized linear constraints of Eq. nlp_updated), sigma_s(x) = sqrt(max(x, 0)^2 + eps^2)

The case uses distinct prices, beta != 1, eps != 0, periods of unequal length, a base rating that
differs from the post-contingency one and a lossy charged line (the two ends carry different
apparent power), so that each slip listed in MUTATIONS changes at least one value.  The mutation
tests plant those slips in a copy of the oracle's source and check that the pins catch every one.
"""
import cmath
import dataclasses
import inspect
import math
import textwrap

import numpy as np
import pytest

import oracle
import synth
from oracle import qg_oracle as Q

EPS = 0.01
BETA = 0.7
PRICES = dict(c_p=900.0, c_q=400.0, c_s=700.0, c_rz=300.0, rho=50.0)

# values per period: v, theta (bus 0 is the reference), p, q, r per device
V = [[1.02, 0.97], [0.99, 1.04]]
TH = [[0.0, -0.35], [0.0, 0.22]]
P = [[0.9, 0.2], [0.5, 0.6]]
QG = [[0.1, -0.05], [-0.2, 0.15]]
R = [[0.3, 0.05], [0.1, 0.25]]
DT = [1.0, 0.5]
LOAD_P = [[0.4, 0.5], [0.3, 0.6]]
LOAD_Q = [[0.1, 0.2], [0.05, 0.1]]
RREQ = [[0.5, 0.1], [0.05, 0.3]]      # [t][zone]
BR = dict(f=1, o=0, r=0.02, x=0.15, bch=0.06)
GEN = dict(bus=[0, 1], zone=[0, 1], a=[0.05, 0.08], b=[20.0, 30.0], cr=[2.0, 4.0], pmax=[1.0, 0.7],
           ramp=[0.3, 0.4])
S_MAX = 0.55
S_MAX_CTG = 5.0


def hand_case():
    arr = np.array
    return synth.Case(
        name="hand2", seed=0, n_bus=2, n_branch=1, n_gen=2, n_zone=2, ref_bus=0,
        br_from=arr([BR["f"]], np.int32), br_to=arr([BR["o"]], np.int32), br_r=arr([BR["r"]]),
        br_x=arr([BR["x"]]), br_b=arr([BR["bch"]]), s_max=arr([S_MAX]), s_max_ctg=arr([S_MAX_CTG]),
        gen_bus=arr(GEN["bus"], np.int32), gen_zone=arr(GEN["zone"], np.int32), cost_a=arr(GEN["a"]),
        cost_b=arr(GEN["b"]), cost_r=arr(GEN["cr"]), pmin=np.zeros(2), pmax=arr(GEN["pmax"]),
        qmin=np.full(2, -1.0), qmax=np.full(2, 1.0), ramp=arr(GEN["ramp"]), vmin=np.full(2, 0.9),
        vmax=np.full(2, 1.1), T=2, dt=arr(DT), load_p=arr(LOAD_P), load_q=arr(LOAD_Q),
        reserve_req=arr(RREQ), bus_zone=arr([0, 1], np.int32), ctg=np.zeros(0, np.int32),
        eps=EPS, beta=BETA, **PRICES)


def hand_point():
    flat = [V, TH, P, QG, R]
    return np.array([val for block in flat for row in block for val in row])


def sa(x, eps):
    return math.sqrt(x * x + eps * eps)


def sr(x, eps):
    m = max(x, 0.0)
    return math.sqrt(m * m + eps * eps)


def end_powers(t):
    """Complex power into the line at both ends, S = V conj(I), textbook pi model."""
    ysr = 1.0 / complex(BR["r"], BR["x"])
    vf = cmath.rect(V[t][BR["f"]], TH[t][BR["f"]])
    vo = cmath.rect(V[t][BR["o"]], TH[t][BR["o"]])
    i_f = ysr * (vf - vo) + 1j * BR["bch"] / 2 * vf
    i_o = ysr * (vo - vf) + 1j * BR["bch"] / 2 * vo
    return vf * i_f.conjugate(), vo * i_o.conjugate()


def hand_terms(eps=EPS):
    out = dict(cost=0.0, zp=0.0, zq=0.0, zs=0.0, zrz=0.0, zhead=0.0, zramp=0.0, zctg=0.0)
    for t in range(2):
        d = DT[t]
        for g in range(2):
            out["cost"] += d * (GEN["a"][g] * P[t][g] ** 2 + GEN["b"][g] * P[t][g] + GEN["cr"][g] * R[t][g])
        sf, so = end_powers(t)
        for i in range(2):
            pi = LOAD_P[t][i]
            qi = LOAD_Q[t][i]
            if BR["f"] == i:
                pi += sf.real
                qi += sf.imag
            if BR["o"] == i:
                pi += so.real
                qi += so.imag
            for g in range(2):
                if GEN["bus"][g] == i:
                    pi -= P[t][g]
                    qi -= QG[t][g]
            out["zp"] += d * PRICES["c_p"] * BETA * sa(pi, eps)
            out["zq"] += d * PRICES["c_q"] * BETA * sa(qi, eps)
        out["zs"] += d * PRICES["c_s"] * BETA * sr(max(abs(sf), abs(so)) - S_MAX, eps)
        for z in range(2):
            have = sum(R[t][g] for g in range(2) if GEN["zone"][g] == z)
            out["zrz"] += d * PRICES["c_rz"] * BETA * sr(RREQ[t][z] - have, eps)
        for g in range(2):
            out["zhead"] += PRICES["rho"] * BETA * sr(P[t][g] + R[t][g] - GEN["pmax"][g], eps)
            if t > 0:
                step = P[t][g] - P[t - 1][g]
                lim = GEN["ramp"][g] * d
                out["zramp"] += PRICES["rho"] * BETA * (sr(step - lim, eps) + sr(-step - lim, eps))
    return out


def terms_match(terms, want, tol=1e-12):
    return all(abs(terms[k] - want[k]) <= tol * max(abs(want[k]), 1e-30) for k in want)


def test_hand_case_activates_every_family():
    """Each family is past its kink somewhere (its hard value, eps = 0, is positive) and the two line
    ends carry different apparent power."""
    sf, so = end_powers(0)
    assert abs(abs(sf) - abs(so)) > 1e-3
    hard = hand_terms(eps=0.0)
    for k in ("cost", "zp", "zq", "zs", "zrz", "zhead", "zramp"):
        assert hard[k] > 1e-3, k


def test_every_term_value_matches_the_hand_computation():
    r = oracle.evaluate(hand_case(), hand_point())
    want = hand_terms()
    for k in want:
        assert abs(r.terms[k] - want[k]) <= 1e-12 * max(abs(want[k]), 1e-30), (k, r.terms[k], want[k])
    assert abs(r.obj - sum(want.values())) <= 1e-12 * abs(r.obj)


def test_hand_case_gradient_against_finite_differences():
    """Every coordinate of the hand case (non-uniform periods, two zones) against central differences."""
    c = hand_case()
    x = hand_point()
    g = oracle.evaluate(c, x).grad
    for i in range(c.n_x):
        h = 1e-6 * max(1.0, abs(x[i]))
        xp = x.copy(); xp[i] += h
        xm = x.copy(); xm[i] -= h
        fd = (oracle.objective(c, xp) - oracle.objective(c, xm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, np.abs(g).max()), (i, fd, g[i])


def test_hard_scoring_values():
    """eps = 0 (the scoring objective): the same sums with the hard |x| and max(x, 0)."""
    r = oracle.evaluate(hand_case(), hand_point(), eps=0.0)
    assert terms_match(r.terms, hand_terms(eps=0.0))


# ------------------------------------------------------------------------------------------------
# planted slips: (function, original text, planted text); each must make a value pin fail
# ------------------------------------------------------------------------------------------------

MUTATIONS = [
    ("evaluate", "u = smax_end - case.s_max[None, :]", "u = smax_end - case.s_max_ctg[None, :]"),
    ("evaluate", "smax_end = np.where(use_fr, sf, st)", "smax_end = np.where(use_fr, st, sf)"),
    ("evaluate", "ws = dt[:, None] * case.c_s * beta", "ws = case.c_s * beta"),
    ("evaluate", "ws = dt[:, None] * case.c_s * beta", "ws = dt[:, None] * case.c_s"),
    ("evaluate", "lim = case.ramp[None, :] * dt[1:, None]", "lim = case.ramp[None, :]"),
    ("evaluate", "lim = case.ramp[None, :] * dt[1:, None]", "lim = case.ramp[None, :] * dt[:-1, None]"),
    ("evaluate", "up = p[1:] - p[:-1] - lim", "up = p[1:] - p[:-1] + lim"),
    ("evaluate", "uh = p + r - case.pmax[None, :] * uon", "uh = case.pmax[None, :] * uon - p - r"),
    ("evaluate", "uh = p + r - case.pmax[None, :] * uon", "uh = p - case.pmax[None, :] * uon"),
    ("evaluate", "uz = case.reserve_req - rz", "uz = rz - case.reserve_req"),
    ("evaluate", "np.add.at(rz.T, case.gen_zone, r.T)", "np.add.at(rz.T, case.gen_zone[::-1], r.T)"),
    ("evaluate", "wz = dt[:, None] * case.c_rz * beta", "wz = dt[:, None] * case.c_s * beta"),
    ("evaluate", "sg * zen + case.cost_r * r)", "sg * zen + case.cost_r * p)"),
    ("evaluate", "(dt[:, None] * (sg * zen + case.cost_r * r))", "((sg * zen + case.cost_r * r))"),
    ("evaluate", "wq = dt[:, None] * case.c_q * beta", "wq = dt[:, None] * case.c_p * beta"),
    ("evaluate", "wr = case.rho * beta", "wr = case.rho"),
    ("energy_cost", "z = case.cost_a * p * p + case.cost_b * p", "z = case.cost_b * p * p + case.cost_a * p"),
    ("soft_abs", "np.sqrt(x * x + eps * eps)", "np.sqrt(x * x + eps)"),
    ("soft_relu", "np.sqrt(m * m + eps * eps)", "np.sqrt(m * m)"),
    ("bus_mismatch", "np.subtract.at(P.T, case.gen_bus, (sg * p).T)", "np.add.at(P.T, case.gen_bus, (sg * p).T)"),
    ("bus_mismatch", "np.add.at(P.T, o, pt.T)", "np.add.at(P.T, f, pt.T)"),
]


def mutant_evaluate(fn, old, new):
    """Q.evaluate running with one slip planted in the source of `fn` (a function of the oracle
    module), compiled into a private copy of the module's namespace; the oracle itself is untouched."""
    ns = dict(vars(Q))
    src = textwrap.dedent(inspect.getsource(getattr(Q, fn)))
    assert src.count(old) == 1, (fn, old)
    exec(compile(src.replace(old, new), f"<mutant {fn}>", "exec"), ns)
    if fn != "evaluate":
        exec(compile(textwrap.dedent(inspect.getsource(Q.evaluate)), "<evaluate>", "exec"), ns)
    return ns["evaluate"]


def test_unmutated_copy_passes():
    ev = mutant_evaluate("evaluate", "wr = case.rho * beta", "wr = case.rho * beta")
    assert terms_match(ev(hand_case(), hand_point()).terms, hand_terms())


@pytest.mark.parametrize("fn,old,new", MUTATIONS, ids=[f"{m[0]}:{m[2][:28]}" for m in MUTATIONS])
def test_planted_slip_is_caught(fn, old, new):
    ev = mutant_evaluate(fn, old, new)
    c = hand_case()
    x = hand_point()
    want = hand_terms()
    caught = not terms_match(ev(c, x).terms, want, tol=1e-9)
    if not caught:  # a slip invisible at eps > 0 must show in the hard scoring objective
        caught = not terms_match(ev(dataclasses.replace(c, eps=0.0), x).terms, hand_terms(eps=0.0), tol=1e-9)
    assert caught, (fn, new)
