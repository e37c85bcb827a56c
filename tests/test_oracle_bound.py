"""Pins of the contingency-aware lower bound (oracle/copperplate.py: contingency_flow_maps,
contingency_bound): the copper-plate relaxation of Sec. III-A plus the DC post-contingency
overloads of Sec. II-E, which are exact (affine) in the dispatch.

- the affine flow maps against brute-force re-solves of every outaged network;
- the LP value against its relaxed objective written out directly (with brute-force contingency
  flows) at the LP's own solution, and that objective at other points never below it (the LP is
  its minimum);
- validity: the bound never exceeds Phi at eps = 0 (random points, the copper-plate start, an
  Adam run of the oracle);
- reductions: no outages, or ratings no dispatch can overload, give the copper-plate bound.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle.copperplate import contingency_bound, contingency_flow_maps, copper_plate


def brute_ctg_flows(case, p):
    """F[t, m, k]: delete branch ctg_k, re-solve the outaged reduced Laplacian with the same
    uniform-slack injections, flows y (theta_f - theta_o); NaN on the outaged branch itself."""
    T, n, M = case.T, case.n_bus, case.n_branch
    y = case.br_x / (case.br_r ** 2 + case.br_x ** 2)
    inj = -case.load_p.copy()
    for g in range(case.n_gen):
        inj[:, case.gen_bus[g]] += p[:, g]
    pbar = inj - inj.mean(axis=1, keepdims=True)
    keep = [i for i in range(n) if i != case.ref_bus]
    F = np.full((T, M, len(case.ctg)), np.nan)
    for kk, k in enumerate(case.ctg):
        Y = np.zeros((n, n))
        for j in range(M):
            if j == k:
                continue
            f, o = case.br_from[j], case.br_to[j]
            Y[f, f] += y[j]; Y[o, o] += y[j]; Y[f, o] -= y[j]; Y[o, f] -= y[j]
        Yr = Y[np.ix_(keep, keep)]
        for t in range(T):
            th = np.zeros(n)
            th[keep] = np.linalg.solve(Yr, pbar[t, keep])
            fl = y * (th[case.br_from] - th[case.br_to])
            fl[k] = np.nan
            F[t, :, kk] = fl
    return F


def relaxed_objective(case, p, r):
    """The bound's objective written out: generator and reserve cost, unserved load at c^p, zonal
    reserve shortfall, headroom and ramp violations (the copper-plate relaxation), plus
    d_t c^s beta max(0, |F| - s^ctg) over every (period, monitored branch, outage)."""
    beta, dt = case.beta, case.dt
    v = (dt[:, None] * (case.cost_a * p * p + case.cost_b * p + case.cost_r * r)).sum()
    v += (dt * case.c_p * beta * np.maximum(0.0, case.load_p.sum(axis=1) - p.sum(axis=1))).sum()
    for z in range(case.n_zone):
        rz = r[:, case.gen_zone == z].sum(axis=1)
        v += (dt * case.c_rz * beta * np.maximum(0.0, case.reserve_req[:, z] - rz)).sum()
    v += case.rho * beta * np.maximum(0.0, p + r - case.pmax).sum()
    if case.T > 1:
        lim = case.ramp[None, :] * dt[1:, None]
        d = p[1:] - p[:-1]
        v += case.rho * beta * (np.maximum(0.0, d - lim) + np.maximum(0.0, -d - lim)).sum()
    if len(case.ctg):
        F = brute_ctg_flows(case, p)
        over = np.nan_to_num(np.maximum(0.0, np.abs(F) - case.s_max_ctg[None, :, None]), nan=0.0)
        v += (dt * case.c_s * beta * over.sum(axis=(1, 2))).sum()
    return v


def dispatch(case, seed):
    rng = np.random.default_rng(seed)
    p = case.pmin + rng.uniform(size=(case.T, case.n_gen)) * (case.pmax - case.pmin)
    r = rng.uniform(size=(case.T, case.n_gen)) * case.pmax * 0.2
    return p, r


@pytest.mark.parametrize("seed", [0, 5])
def test_flow_maps_match_brute_force_resolves(seed):
    c = synth.tiny(seed)
    J, f0, Lo = contingency_flow_maps(c)
    p, _ = dispatch(c, 3)
    f = p @ J.T + f0
    F = f[:, :, None] + Lo[None, :, :] * f[:, c.ctg][:, None, :]
    Fb = brute_ctg_flows(c, p)
    ok = ~np.isnan(Fb)
    assert np.allclose(F[ok], Fb[ok], rtol=1e-10, atol=1e-12)
    assert np.all(np.isnan(Fb[:, c.ctg, np.arange(len(c.ctg))]))
    # base flows of the maps against the oracle's own base solve
    _, fo = oracle.dc_base_flows(c, oracle.dc_network(c), oracle.dc_injections(c, p)[1])
    assert np.allclose(f, fo, rtol=1e-12, atol=1e-12)


@pytest.fixture(scope="module")
def tiny_bound():
    c = synth.tiny()
    return c, contingency_bound(c)


def test_lp_value_is_its_relaxed_objective_at_its_solution(tiny_bound):
    c, (b, p, r, nS) = tiny_bound
    assert nS > 0
    assert abs(relaxed_objective(c, p, r) - b) <= 1e-7 * b


def test_relaxed_objective_never_falls_below_the_bound(tiny_bound):
    c, (b, p, r, _) = tiny_bound
    _, pc, rc = copper_plate(c)
    assert relaxed_objective(c, pc, rc) >= b * (1 - 1e-9)
    for seed in range(6):
        pr, rr = dispatch(c, seed)
        assert relaxed_objective(c, pr, rr) >= b * (1 - 1e-9)
    rng = np.random.default_rng(7)
    for _ in range(6):  # small moves around the LP solution stay above it (convexity, optimum)
        pp = np.clip(p + 0.01 * rng.standard_normal(p.shape), c.pmin, c.pmax)
        assert relaxed_objective(c, pp, r) >= b * (1 - 1e-9)


def test_bound_is_valid_and_above_the_copper_plate_bound(tiny_bound):
    c, (b, p, r, _) = tiny_bound
    cp, pc, rc = copper_plate(c)
    assert b >= cp * (1 - 1e-12)
    lo, hi = oracle.box(c)
    pts = [c.flat_start(pc, rc), c.flat_start(p, r)] + [synth.random_point(c, s) for s in range(4)]
    x = np.clip(c.flat_start(pc, rc), lo, hi)
    m, v = np.zeros_like(x), np.zeros_like(x)
    for i in range(1, 61):
        res = oracle.evaluate(c, x)
        x, m, v = oracle.adam_step(x, m, v, res.grad, i, 2e-3, 0.9, 0.999, 1e-8, lo, hi)
        if i % 20 == 0:
            pts.append(x.copy())
    for xp in pts:
        assert oracle.evaluate(c, xp, eps=0.0, want_grad=False).obj >= b * (1 - 1e-12)


def test_reductions_to_the_copper_plate_bound():
    c = synth.tiny()
    cp = copper_plate(c)[0]
    b0, _, _, n0 = contingency_bound(dataclasses.replace(c, ctg=np.zeros(0, np.int32)))
    assert n0 == 0 and b0 == pytest.approx(cp, rel=1e-12)
    loose = dataclasses.replace(c, s_max_ctg=np.full(c.n_branch, 1e3))
    bl, _, _, nl = contingency_bound(loose)
    assert nl == 0 and bl == pytest.approx(cp, rel=1e-9)


def test_bound_on_a_meshed_73_bus_grid():
    """On the 73-bus grid the contingency overloads are avoidable at little cost: the bound stays
    valid and lies just above the copper-plate bound."""
    c = synth.mid()
    cp, pc, rc = copper_plate(c)
    b, p, r, nS = contingency_bound(c)
    assert nS > 0 and cp * (1 - 1e-12) <= b <= 1.05 * cp
    lo, hi = oracle.box(c)
    for xp in [c.flat_start(pc, rc), c.flat_start(p, r)] + [synth.random_point(c, s) for s in range(3)]:
        assert oracle.evaluate(c, np.clip(xp, lo, hi), eps=0.0, want_grad=False).obj >= b * (1 - 1e-12)


def test_device_models_and_phase_shifters_are_refused():
    c = synth.tiny()
    for bad in (synth.with_block_bids(c, 3, 0.3, 1), synth.with_commitment(c, seed=1)):
        with pytest.raises(ValueError):
            copper_plate(bad)
        with pytest.raises(ValueError):
            contingency_bound(bad)
    with pytest.raises(ValueError):
        contingency_bound(synth.with_transformers(c, 0.3, 4))


def test_stored_time_to_target_bounds_match_the_oracle():
    """tests/golden/rt617_ttt_bounds.json (written by make_ttt_bounds.py) holds the bounds that the
    time-to-target comparison states its target against: recompute both bounds of the quickest
    profile (the contingency-aware LP takes about 40 s there) and check the ordering of the rest."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rt617_ttt_bounds.json")
    rows = json.load(open(path))["rows"]
    base = synth.rt617()
    prof = synth.load_profiles(base, len(rows), 5001)
    for r in rows:
        assert r["contingency_bound"] >= r["copper_plate"] > 0
    quick = min(rows, key=lambda r: r["triples"])
    c = synth.with_loads(base, prof[quick["profile"]])
    assert copper_plate(c)[0] == pytest.approx(quick["copper_plate"], rel=1e-9)
    assert contingency_bound(c)[0] == pytest.approx(quick["contingency_bound"], rel=1e-7)
