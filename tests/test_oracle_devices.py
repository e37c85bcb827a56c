"""Pins of the oracle's device models: block bids (Example 3), consumers (the market-surplus sign and
Example 4's balance sign) and relaxed on/off status with startup and shutdown (Example 2).

Each is checked against a formulation the paper states separately from the one the oracle codes:
the block LP of Example 3 against its max/min form, the evolution equations of Example 2 against
their max form, a consumer held fixed against the same draw written as fixed load, and commitment
at u = 1 against the case without it."""
import dataclasses

import numpy as np
import pytest
from scipy.optimize import linprog

import oracle
import synth
from oracle import qg_oracle as Q


def _smooth(case, eps=0.05):
    return dataclasses.replace(case, eps=eps)


def _fd(case, x, idx, h=1e-6):
    out = np.empty(len(idx))
    for n_, i in enumerate(idx):
        hh = h * max(1.0, abs(x[i]))
        xp = x.copy(); xp[i] += hh
        xm = x.copy(); xm[i] -= hh
        out[n_] = (oracle.objective(case, xp) - oracle.objective(case, xm)) / (2 * hh)
    return out


def _bids(seed=1):
    return synth.with_block_bids(synth.tiny(), n_blocks=3, cons_frac=0.3, seed=seed)


def _one_device(price, width, p):
    """energy_cost of a single device with the given blocks at the dispatch values p (1-D)."""
    L = len(price)
    c = dataclasses.replace(synth.tiny(), n_gen=1, cost_a=np.zeros(1), cost_b=np.zeros(1),
                            blk_price=np.asarray(price, float).reshape(1, L),
                            blk_width=np.asarray(width, float).reshape(1, L))
    z, dz = oracle.energy_cost(c, np.asarray(p, float).reshape(-1, 1))
    return z[:, 0], dz[:, 0]


def _block_lp(price, width, p, maximize):
    """Example 3's first form: blocks 0 <= p_m <= w_m summing to p, cost (or value) sum c_m p_m."""
    c = -np.asarray(price) if maximize else np.asarray(price)
    res = linprog(c, A_eq=np.ones((1, len(price))), b_eq=[p], bounds=list(zip([0.0] * len(width), width)),
                  method="highs")
    assert res.status == 0
    return -res.fun if maximize else res.fun


# --------------------------------------------------------------------------------------------
# Example 3: block bids
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_block_cost_equals_the_block_lp(seed):
    """Convex costs (rising prices, minimized) and concave values (falling prices, maximized): the
    max/min form equals the optimum of the block LP at every dispatch inside the blocks."""
    rng = np.random.default_rng(seed)
    L = int(rng.integers(1, 6))
    width = rng.uniform(0.1, 2.0, L)
    rising = np.cumsum(rng.uniform(0.5, 10.0, L))
    for price, maximize in ((rising, False), (rising[::-1].copy(), True)):
        ps = rng.uniform(0.0, width.sum(), 16)
        z, _ = _one_device(price, width, ps)
        for pv, zv in zip(ps, z):
            assert abs(zv - _block_lp(price, width, pv, maximize)) <= 1e-9 * max(1.0, abs(zv))


def test_block_cost_right_derivative_at_and_between_edges():
    """The derivative is the right derivative of the block LP: the entered block's price, at block
    edges too, and 0 past the last block."""
    price, width = [10.0, 20.0, 30.0], [1.0, 2.0, 1.0]
    p = np.array([0.0, 0.5, 1.0, 2.5, 3.0, 3.5, 4.0, 4.5])
    z, dz = _one_device(price, width, p)
    np.testing.assert_allclose(z, [0.0, 5.0, 10.0, 40.0, 50.0, 65.0, 80.0, 80.0], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(dz, [10.0, 10.0, 20.0, 20.0, 30.0, 30.0, 0.0, 0.0])
    h = 1e-3  # every point is at least 0.5 from the next block edge; well above the LP tolerances
    for pv, dv in zip(p, dz):
        if pv < 4.0:
            right = (_block_lp(price, width, pv + h, False) - _block_lp(price, width, pv, False)) / h
            assert abs(right - dv) <= 1e-5 * 30


def test_single_block_is_the_linear_cost():
    c = synth.tiny()
    p = synth.random_point(c, 2)[2 * c.T * c.n_bus:][:c.T * c.n_gen].reshape(c.T, c.n_gen)
    lin = dataclasses.replace(c, cost_a=np.zeros(c.n_gen))
    blk = dataclasses.replace(lin, blk_price=c.cost_b[:, None].copy(), blk_width=c.pmax[:, None].copy())
    z0, d0 = oracle.energy_cost(lin, p)
    z1, d1 = oracle.energy_cost(blk, p)
    np.testing.assert_allclose(z1, z0, rtol=1e-14, atol=0)
    np.testing.assert_array_equal(d1, d0)


# --------------------------------------------------------------------------------------------
# consumers: Example 4's balance sign and the market-surplus sign
# --------------------------------------------------------------------------------------------

def _as_fixed_load(c, x):
    """The case with its consumers removed and their draw at x added to the fixed load, and the
    matching point."""
    v, th, p, q, r = oracle.unpack(c, x)
    cons = np.asarray(c.dev_cons, bool)
    keep = ~cons
    load_p, load_q = c.load_p.copy(), c.load_q.copy()
    np.add.at(load_p.T, c.gen_bus[cons], p[:, cons].T)
    np.add.at(load_q.T, c.gen_bus[cons], q[:, cons].T)
    sub = lambda a: a[keep]
    c2 = dataclasses.replace(
        c, n_gen=int(keep.sum()), gen_bus=sub(c.gen_bus), gen_zone=sub(c.gen_zone), cost_a=sub(c.cost_a),
        cost_b=sub(c.cost_b), cost_r=sub(c.cost_r), pmin=sub(c.pmin), pmax=sub(c.pmax), qmin=sub(c.qmin),
        qmax=sub(c.qmax), ramp=sub(c.ramp), load_p=load_p, load_q=load_q, dev_cons=sub(cons),
        blk_price=c.blk_price[keep], blk_width=c.blk_width[keep])
    x2 = oracle.pack(v, th, p[:, keep], q[:, keep], r[:, keep])
    return c2, x2, p[:, cons]


@pytest.mark.parametrize("seed", [1, 4])
def test_consumer_draw_equals_the_same_fixed_load(seed):
    """Balance, thermal and contingency terms (and the v, theta gradient) see a consumer exactly
    as fixed load of the same size; the cost differs by the consumer's value, which it earns."""
    c = _bids(seed)
    assert c.n_cons >= 2
    x = synth.random_point(c, seed + 10)
    c2, x2, pc = _as_fixed_load(c, x)
    a, b = oracle.evaluate(c, x), oracle.evaluate(c2, x2)
    for k in ("zp", "zq", "zs", "zrz", "zctg"):
        assert abs(a.terms[k] - b.terms[k]) <= 1e-10 * max(1.0, abs(b.terms[k])), k
    cons = np.asarray(c.dev_cons, bool)
    L = c.blk_price.shape[1]
    value = 0.0
    for j, g in enumerate(np.flatnonzero(cons)):
        for t in range(c.T):
            value += c.dt[t] * _block_lp(c.blk_price[g], c.blk_width[g], pc[t, j], True) if L else 0.0
    assert abs((a.terms["cost"] - b.terms["cost"]) + value) <= 1e-9 * max(1.0, value)
    n = c.T * c.n_bus
    np.testing.assert_allclose(a.grad[:2 * n], b.grad[:2 * n], rtol=0, atol=1e-9 * np.abs(b.grad).max())


@pytest.mark.parametrize("seed", [1, 2])
def test_fd_gradient_bids_consumers_commitment_all_coordinates(seed):
    c = _smooth(synth.with_commitment(_bids(seed), seed=seed))
    x = synth.random_point(c, seed + 20)
    g = oracle.evaluate(c, x).grad
    fd = _fd(c, x, np.arange(c.n_x))
    scale = np.abs(g).max()
    assert np.max(np.abs(fd - g)) <= 1e-7 * scale, np.max(np.abs(fd - g)) / scale
    assert np.abs(g[c.offset_u():]).max() > 1e-4 * scale  # the on-status coordinates carry gradient


def test_box_of_consumers_and_commitment():
    c = synth.with_commitment(_bids(1), seed=1)
    lo, hi = oracle.box(c)
    _, _, plo, qlo, rlo = oracle.unpack(c, lo)
    _, _, phi_, qhi, rhi = oracle.unpack(c, hi)
    cons = np.asarray(c.dev_cons, bool)
    assert np.all(rhi[:, cons] == 0) and np.all(rhi[:, ~cons] == c.pmax[~cons])
    assert np.all(plo == 0) and np.all(qlo <= 0) and np.all(qhi >= 0)
    assert np.all(oracle.unpack_u(c, lo) == 0) and np.all(oracle.unpack_u(c, hi) == 1)


# --------------------------------------------------------------------------------------------
# Example 2: on/off status, startup and shutdown
# --------------------------------------------------------------------------------------------

def _no_commit(c, x):
    c0 = dataclasses.replace(c, commit=False)
    return c0, x[:c0.n_x]


def _evolution_lp(u, u0, csu, csd):
    """Example 2's evolution equations as an LP over startup / shutdown indicators in [0, 1]:
    su_t - sd_t = u_t - u_{t-1}, su_t + sd_t <= 1, minimizing c_su su + c_sd sd."""
    T = len(u)
    du = np.diff(np.concatenate([[u0], u]))
    A_eq = np.hstack([np.eye(T), -np.eye(T)])
    A_ub = np.hstack([np.eye(T), np.eye(T)])
    res = linprog(np.concatenate([np.full(T, csu), np.full(T, csd)]), A_ub=A_ub, b_ub=np.ones(T), A_eq=A_eq,
                  b_eq=du, bounds=[(0.0, 1.0)] * (2 * T), method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("seed", [0, 3])
def test_startup_shutdown_cost_equals_the_evolution_lp(seed):
    c = synth.with_commitment(synth.tiny(), seed=seed)
    x = synth.random_point(c, seed + 5)
    u = oracle.unpack_u(c, x)
    c0, x0 = _no_commit(c, x)
    extra = oracle.evaluate(c, x).terms["cost"] - oracle.evaluate(c0, x0).terms["cost"]
    want = float((c.dt[:, None] * c.c_on * u).sum())
    for g in range(c.n_gen):
        want += _evolution_lp(u[:, g], c.u_init[g], c.c_su[g], c.c_sd[g])
    assert abs(extra - want) <= 1e-9 * want


def test_binary_status_charges_each_start_and_stop_once():
    c = synth.with_commitment(synth.tiny(), seed=5)
    rng = np.random.default_rng(0)
    x = synth.random_point(c, 1)
    o = c.offset_u()
    u = (rng.uniform(size=(c.T, c.n_gen)) < 0.5).astype(float)
    x[o:] = u.ravel()
    c0, x0 = _no_commit(c, x)
    extra = oracle.evaluate(c, x).terms["cost"] - oracle.evaluate(c0, x0).terms["cost"]
    want = 0.0
    for g in range(c.n_gen):
        prev = c.u_init[g]
        for t in range(c.T):
            want += c.dt[t] * c.c_on[g] * u[t, g]
            if prev == 0 and u[t, g] == 1:
                want += c.c_su[g]
            if prev == 1 and u[t, g] == 0:
                want += c.c_sd[g]
            prev = u[t, g]
    assert abs(extra - want) <= 1e-12 * want


def test_commitment_at_u_one_reduces_to_the_plain_case():
    """With every device on (u = 1, u_init = 1, no on cost) and p, q inside their limits, the
    u-scaled limits are slack: at eps = 0 the objective and every shared gradient coordinate equal
    those of the case without commitment, and the u gradient is -pmax times the headroom weight."""
    c = synth.with_commitment(synth.tiny(), seed=2)
    c = dataclasses.replace(c, c_on=np.zeros(c.n_gen), u_init=np.ones(c.n_gen))
    x = synth.random_point(c, 4)
    x[c.offset_u():] = 1.0
    c0, x0 = _no_commit(c, x)
    a, b = oracle.evaluate(c, x, eps=0.0), oracle.evaluate(c0, x0, eps=0.0)
    assert abs(a.obj - b.obj) <= 1e-12 * abs(b.obj)
    np.testing.assert_array_equal(a.grad[:c0.n_x], b.grad)
    _, _, p, _, r = oracle.unpack(c, x)
    head = (p + r - c.pmax > 0) * c.rho * c.beta
    np.testing.assert_allclose(oracle.unpack_u(c, a.grad), c.c_su * 0 - c.pmax * head, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------------------------
# planted mistakes
# --------------------------------------------------------------------------------------------

def test_planted_unsigned_consumer_injection_is_caught(monkeypatch):
    c = _bids(1)
    x = synth.random_point(c, 11)
    c2, x2, _ = _as_fixed_load(c, x)

    def bad(case, p):
        inj = -case.load_p.copy()
        np.add.at(inj.T, case.gen_bus, p.T)  # consumers counted as supply
        return inj, inj - inj.mean(axis=1, keepdims=True)
    monkeypatch.setattr(Q, "dc_injections", bad)
    a, b = oracle.evaluate(c, x), oracle.evaluate(c2, x2)
    assert abs(a.terms["zctg"] - b.terms["zctg"]) > 1e-6 * b.terms["zctg"]


def test_planted_left_derivative_at_block_edges_is_caught(monkeypatch):
    orig = Q.energy_cost

    def bad(case, p):
        z, dz = orig(case, p)
        W = case.blk_width
        if W.size:
            edge = np.isclose(p, W[:, 0][None, :])
            dz = np.where(edge, case.blk_price[:, 0][None, :], dz)
        return z, dz
    monkeypatch.setattr(Q, "energy_cost", bad)
    monkeypatch.setattr(oracle, "energy_cost", bad)
    with pytest.raises(AssertionError):
        test_block_cost_right_derivative_at_and_between_edges()
