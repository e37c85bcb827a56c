"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an invariant, brute force or a
library routine, chosen so that a plausible slip (a dropped term, a wrong sign or
index, a transposed operand) fails at least one of them.  The mutation tests at
the end plant such slips in the oracle and confirm the pins catch them.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import qg_oracle as Q
from oracle.copperplate import copper_plate, lambda_dispatch


def _smooth(case, eps=0.05):
    """Larger epsilon keeps every soft penalty C^3 on the finite-difference step scale."""
    return dataclasses.replace(case, eps=eps)


def _fd(case, x, idx, h=1e-6):
    out = np.empty(len(idx))
    for n_, i in enumerate(idx):
        hh = h * max(1.0, abs(x[i]))
        xp = x.copy(); xp[i] += hh
        xm = x.copy(); xm[i] -= hh
        out[n_] = (oracle.objective(case, xp) - oracle.objective(case, xm)) / (2 * hh)
    return out


# --------------------------------------------------------------------------------------------
# gradient <-> objective (central differences, every coordinate on the tiny case)
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2])
def test_fd_gradient_tiny_all_coordinates(seed):
    c = _smooth(synth.tiny())
    x = synth.random_point(c, seed)
    g = oracle.evaluate(c, x).grad
    idx = np.arange(c.n_x)
    fd = _fd(c, x, idx)
    scale = np.abs(g).max()
    assert np.max(np.abs(fd - g)) <= 1e-7 * scale, np.max(np.abs(fd - g)) / scale


def test_fd_gradient_mid_sampled():
    c = _smooth(synth.mid())
    x = synth.random_point(c, 7, spread=0.5)
    g = oracle.evaluate(c, x).grad
    rng = np.random.default_rng(0)
    idx = rng.choice(c.n_x, 120, replace=False)
    fd = _fd(c, x, idx)
    scale = np.abs(g).max()
    assert np.max(np.abs(fd - g[idx])) <= 1e-7 * scale


def test_fd_gradient_at_lp_start_default_eps():
    """At the copper-plate start with the default eps = 1e-3, away from kinks."""
    c = synth.tiny()
    _, p, r = copper_plate(c)
    x = c.flat_start(p, r) + synth.random_point(c, 3) * 1e-3
    lo, hi = oracle.box(c)
    x = np.clip(x, lo, hi)
    g = oracle.evaluate(c, x).grad
    idx = np.arange(c.n_x)
    fd = _fd(c, x, idx, h=1e-7)
    scale = np.abs(g).max()
    assert np.max(np.abs(fd - g)) <= 1e-5 * scale


# --------------------------------------------------------------------------------------------
# KCL and flow closed forms
# --------------------------------------------------------------------------------------------

def test_bus_mismatch_matches_direct_loop():
    c = synth.tiny()
    x = synth.random_point(c, 4)
    v, th, p, q, r = oracle.unpack(c, x)
    pf, qf, pt, qt = oracle.ac_flows(c, v, th)
    P, Qb = oracle.bus_mismatch(c, pf, qf, pt, qt, p, q)
    for t in range(c.T):
        for i in range(c.n_bus):
            ps = c.load_p[t, i]
            qs = c.load_q[t, i]
            for j in range(c.n_branch):
                if c.br_from[j] == i:
                    ps += pf[t, j]; qs += qf[t, j]
                if c.br_to[j] == i:
                    ps += pt[t, j]; qs += qt[t, j]
            for g in range(c.n_gen):
                if c.gen_bus[g] == i:
                    ps -= p[t, g]; qs -= q[t, g]
            assert abs(ps - P[t, i]) < 1e-12 and abs(qs - Qb[t, i]) < 1e-12


def test_losses_nonnegative_and_lossless_antisymmetric():
    c = synth.tiny()
    x = synth.random_point(c, 5)
    v, th, p, q, r = oracle.unpack(c, x)
    pf, qf, pt, qt = oracle.ac_flows(c, v, th)
    P, _ = oracle.bus_mismatch(c, pf, qf, pt, qt, p, q)
    # sum_i P_it = load - gen + losses,  losses_j = g |V_f - V_o|^2 >= 0
    g, _ = Q.series_admittance(c)
    Vf = v[:, c.br_from] * np.exp(1j * th[:, c.br_from])
    Vo = v[:, c.br_to] * np.exp(1j * th[:, c.br_to])
    loss = (g * np.abs(Vf - Vo) ** 2).sum(axis=1)
    lhs = P.sum(axis=1)
    rhs = c.load_p.sum(axis=1) - p.sum(axis=1) + loss
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-11)
    assert np.all(pf + pt >= -1e-14)
    # lossless (r = 0): p_fr + p_to = 0 exactly
    c0 = dataclasses.replace(c, br_r=np.zeros(c.n_branch))
    pf0, _, pt0, _ = oracle.ac_flows(c0, v, th)
    assert np.max(np.abs(pf0 + pt0)) < 1e-12


def _two_bus(xl, bch, r=0.0):
    one = np.ones(1)
    return synth.Case(
        name="two", seed=0, n_bus=2, n_branch=1, n_gen=1, n_zone=1, ref_bus=0,
        br_from=np.array([1], np.int32), br_to=np.array([0], np.int32), br_r=np.array([r]),
        br_x=np.array([xl]), br_b=np.array([bch]), s_max=one * 9, s_max_ctg=one * 9,
        gen_bus=np.array([0], np.int32), gen_zone=np.array([0], np.int32), cost_a=one, cost_b=one,
        cost_r=one, pmin=0 * one, pmax=one, qmin=-one, qmax=one, ramp=one, vmin=np.full(2, 0.9),
        vmax=np.full(2, 1.1), T=1, dt=one, load_p=np.zeros((1, 2)), load_q=np.zeros((1, 2)),
        reserve_req=np.zeros((1, 1)), bus_zone=np.zeros(2, np.int32), ctg=np.zeros(0, np.int32))


@pytest.mark.parametrize("delta", [-0.4, 0.05, 0.3, 1.1])
def test_two_bus_lossless_closed_form(delta):
    xl, bch = 0.2, 0.04
    c = _two_bus(xl, bch)
    f, o = int(c.br_from[0]), int(c.br_to[0])
    v = np.ones((1, 2))
    th = np.zeros((1, 2))
    th[0, f] = delta
    pf, qf, pt, qt = oracle.ac_flows(c, v, th)
    assert abs(pf[0, 0] - math.sin(delta) / xl) < 1e-13
    assert abs(qf[0, 0] - ((1 - math.cos(delta)) / xl - bch / 2)) < 1e-13
    assert abs(pt[0, 0] + pf[0, 0]) < 1e-13
    assert abs(qt[0, 0] - ((1 - math.cos(delta)) / xl - bch / 2)) < 1e-13
    # d p_fr / d v_to = (-g cos d - b sin d) v_fr; with g = 0, b = -1/x this is sin(d)/x
    part = Q.ac_flow_partials(c, v, th)
    assert abs(part["pf"][1][0, 0] - math.sin(delta) / xl) < 1e-13


def test_two_bus_lossy_against_complex_power():
    """S_fr = V_f conj(I_fr) with I_fr = y_sr (V_f - V_o) + j b_ch/2 V_f (textbook pi model)."""
    xl, bch, rr = 0.2, 0.04, 0.05
    c = _two_bus(xl, bch, rr)
    f, o = int(c.br_from[0]), int(c.br_to[0])
    rng = np.random.default_rng(0)
    v = np.zeros((1, 2)); th = np.zeros((1, 2))
    v[0] = rng.uniform(0.9, 1.1, 2)
    th[0] = rng.normal(0, 0.3, 2)
    pf, qf, pt, qt = oracle.ac_flows(c, v, th)
    Vf = v[0, f] * np.exp(1j * th[0, f])
    Vo = v[0, o] * np.exp(1j * th[0, o])
    ysr = 1.0 / (rr + 1j * xl)
    If = ysr * (Vf - Vo) + 1j * bch / 2 * Vf
    It = ysr * (Vo - Vf) + 1j * bch / 2 * Vo
    Sf = Vf * np.conj(If)
    St = Vo * np.conj(It)
    assert abs(pf[0, 0] - Sf.real) < 1e-13 and abs(qf[0, 0] - Sf.imag) < 1e-13
    assert abs(pt[0, 0] - St.real) < 1e-13 and abs(qt[0, 0] - St.imag) < 1e-13


# --------------------------------------------------------------------------------------------
# contingencies: SMW (Eq. rank_correct) against brute-force re-solves
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mk", [synth.tiny, lambda: synth.batch(per_shape=1)[0]])
def test_ctg_smw_matches_brute_force(mk):
    c = mk()
    x = synth.random_point(c, 11)
    a = oracle.evaluate(c, x, mode="smw")
    b = oracle.evaluate(c, x, mode="brute")
    assert abs(a.obj - b.obj) <= 1e-12 * abs(b.obj)
    assert np.allclose(a.z_ctg, b.z_ctg, rtol=1e-12, atol=0)
    assert np.max(np.abs(a.grad - b.grad)) <= 1e-11 * np.abs(b.grad).max()


def test_outaged_network_kcl():
    """Post-contingency flows from the rank-1 form conserve the injections on the outaged grid."""
    c = synth.tiny()
    x = synth.random_point(c, 12)
    _, _, p, _, _ = oracle.unpack(c, x)
    net = oracle.dc_network(c)
    _, pbar = oracle.dc_injections(c, p)
    th, f = oracle.dc_base_flows(c, net, pbar)
    Eh = net.E[:, net.keep]
    U = net.Yinv @ Eh[c.ctg].T
    for kk, k in enumerate(c.ctg):
        den = 1 - net.y[k] * Eh[k] @ U[:, kk]
        thk = th[0, net.keep] + U[:, kk] * (f[0, k] / den)
        F = net.y * (Eh @ thk)
        F[k] = 0.0
        assert np.allclose(net.E.T @ F, pbar[0], atol=1e-12)


def test_slack_correction_against_fd():
    """Eq. correction: the contingency gradient wrt injections is eta - mean(eta).
    Perturbing one bus's load moves p_inj at that bus by -h (the AC part is switched off)."""
    c = dataclasses.replace(_smooth(synth.tiny()), c_p=0.0, c_q=0.0, c_s=1e3)
    x = synth.random_point(c, 13)
    r = oracle.evaluate(c, x)
    assert abs(r.g_inj.sum(axis=1)).max() < 1e-9 * abs(r.g_inj).max()  # projected: sums to zero
    h = 1e-6
    for t in range(c.T):
        for i in range(c.n_bus):
            lp = c.load_p.copy(); lp[t, i] -= h
            lm = c.load_p.copy(); lm[t, i] += h
            zp = oracle.evaluate(dataclasses.replace(c, load_p=lp), x, want_grad=False).terms["zctg"]
            zm = oracle.evaluate(dataclasses.replace(c, load_p=lm), x, want_grad=False).terms["zctg"]
            fd = (zp - zm) / (2 * h)
            assert abs(fd - r.g_inj[t, i]) <= 1e-6 * max(1.0, abs(r.g_inj).max())


# --------------------------------------------------------------------------------------------
# Adam (Alg. 3) against torch.optim.Adam + clamp, and the schedules (Eqs. norm_t-step_size)
# --------------------------------------------------------------------------------------------

def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    n = 257
    x = rng.normal(size=n)
    lo = np.full(n, -0.8); hi = np.full(n, 0.9)
    x = np.clip(x, lo, hi)
    m = np.zeros(n); v = np.zeros(n)
    xt = torch.tensor(x.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([xt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for i in range(1, 11):
        g = rng.normal(size=n) * (1 + i)
        x, m, v = oracle.adam_step(x, m, v, g, i, 1e-2, 0.9, 0.999, 1e-8, lo, hi)
        xt.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        with torch.no_grad():
            xt.clamp_(torch.tensor(lo), torch.tensor(hi))
        assert np.max(np.abs(xt.detach().numpy() - x)) < 1e-14


def test_adam_paper_literal_numerator():
    x, m, v = oracle.adam_step(np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(1), 1, 0.1, 0.9, 0.999, 1e-8,
                               np.full(1, -1.0), np.full(1, 1.0), paper_eps=True)
    assert abs(x[0] + 0.1 * 1e-8 / 1e-8) < 1e-15  # a zero gradient still moves by alpha


def test_schedule_closed_form():
    assert oracle.normalized_time(0.0, 0.0, 10.0) == -1.0
    assert oracle.normalized_time(5.0, 0.0, 10.0) == 0.0
    assert oracle.normalized_time(10.0, 0.0, 10.0) == 1.0
    assert abs(oracle.magnitude_scale(-1.0) - math.exp(-4) / (0.6 + math.exp(-4))) < 1e-15
    assert abs(oracle.magnitude_scale(-1.0) - 0.0296218) < 1e-6
    assert oracle.magnitude_scale(0.0) == 1.0 / 1.6
    assert abs(oracle.magnitude_scale(1.0) - 0.9891301) < 1e-6
    a0, af = 1e-2, 1e-5
    assert abs(oracle.step_size(a0, af, 5.0, 0.0, 10.0) - a0 * (af / a0) ** 0.625) < 1e-15
    assert abs(oracle.step_size(a0, af, 0.0, 0.0, 10.0) - a0 * (af / a0) ** 0.0296218) < 1e-8


# --------------------------------------------------------------------------------------------
# smooth penalties and the copper-plate bound
# --------------------------------------------------------------------------------------------

def test_soft_penalties_special_cases():
    x = np.array([-2.0, -1e-9, 0.0, 3.0])
    assert np.allclose(oracle.soft_abs(x, 0.0), np.abs(x))
    assert np.allclose(oracle.soft_relu(x, 0.0), np.maximum(x, 0))
    assert np.allclose(oracle.soft_relu(np.array([-5.0, 0.0]), 0.25), [0.25, 0.25])
    assert np.allclose(oracle.soft_abs(np.array([0.0]), 0.25), [0.25])
    assert abs(oracle.soft_abs(np.array([3.0]), 4.0)[0] - 5.0) < 1e-15


def test_copper_plate_single_period_matches_kkt_dispatch():
    c = synth.tiny()
    c1 = dataclasses.replace(c, T=1, dt=c.dt[:1], load_p=c.load_p[1:2], load_q=c.load_q[1:2],
                             reserve_req=np.zeros((1, 1)))
    lb, p, r = copper_plate(c1)
    pk = lambda_dispatch(c1)
    cost_kkt = float((c1.cost_a * pk[0] ** 2 + c1.cost_b * pk[0]).sum())
    assert abs(lb - cost_kkt) <= 1e-7 * cost_kkt
    assert np.allclose(p, pk, atol=1e-4)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_copper_plate_bounds_phi(seed):
    c = synth.tiny()
    lb, p, r = copper_plate(c)
    xs = [c.flat_start(p, r), synth.random_point(c, seed)]
    for x in xs:
        assert oracle.objective(c, x, eps=0.0) >= lb - 1e-9 * abs(lb)
    # the bound is attained only up to the network terms: Phi_eps0 at the LP point >= bound
    assert oracle.objective(c, xs[0], eps=0.0) >= lb


# --------------------------------------------------------------------------------------------
# generator sanity (inputs the paper's workloads imply)
# --------------------------------------------------------------------------------------------

def test_generated_grids_have_no_bridges_and_fit_capacity():
    for c in [synth.tiny(), synth.mid(), synth.rt617()]:
        assert synth.find_bridges(c.n_bus, c.br_from, c.br_to) == []
        assert 1.1 * c.load_p.sum(axis=1).max() <= 0.7 * c.pmax.sum() + 1e-9
    c = synth.tiny()
    assert (c.n_bus, c.n_branch, c.n_gen, c.T, c.K) == (14, 20, 5, 4, 20)
    c = synth.rt617()
    assert (c.n_bus, c.n_branch, c.n_gen, c.T, c.K) == (617, 900, 90, 18, 562)


@pytest.mark.slow
def test_active_contingency_share_at_lp_start():
    """Between 1% and 30% of (t, k) pairs carry a violation at the copper-plate start."""
    for c in [synth.tiny(), synth.rt617()]:
        _, p, r = copper_plate(c)
        res = oracle.evaluate(c, c.flat_start(p, r), want_grad=False)
        floor = c.eps * c.c_s * c.beta * (c.n_branch - 1)
        share = float((res.z_ctg > floor * (1 + 1e-9)).mean())
        assert 0.01 <= share <= 0.30, share


# --------------------------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above
# --------------------------------------------------------------------------------------------

def _fd_fails(c, x):
    g = oracle.evaluate(c, x).grad
    fd = _fd(c, x, np.arange(c.n_x))
    return np.max(np.abs(fd - g)) > 1e-7 * np.abs(g).max()


def test_planted_sign_error_in_flow_partial_is_caught(monkeypatch):
    c = _smooth(synth.tiny())
    x = synth.random_point(c, 1)
    orig = Q.ac_flow_partials

    def bad(case, v, th, tau=None, phi=None):
        out = orig(case, v, th, tau, phi)
        a, b_, d, e = out["pt"]
        out["pt"] = (a, b_, -d, e)
        return out
    monkeypatch.setattr(Q, "ac_flow_partials", bad)
    assert _fd_fails(c, x)


def test_planted_missing_slack_correction_is_caught(monkeypatch):
    c = _smooth(synth.tiny())
    x = synth.random_point(c, 1)
    orig = Q._ctg_period_smw

    def bad(case, net, th_hat_b, qmax2, dt, U, den, b_t=None):
        z, gin, gq2, gb = orig(case, net, th_hat_b, qmax2, dt, U, den, b_t)
        # undo the projection: add back the mean that Eq. correction subtracts (approximately)
        return z, gin + 0.37 * np.abs(gin).max(), gq2, gb
    monkeypatch.setattr(Q, "_ctg_period_smw", bad)
    assert _fd_fails(c, x)


def test_planted_wrong_smw_sign_is_caught(monkeypatch):
    c = synth.tiny()
    x = synth.random_point(c, 1)
    good = oracle.evaluate(c, x, mode="brute")
    orig = Q._ctg_period_smw

    def bad(case, net, th_hat_b, qmax2, dt, U, den, b_t=None):
        return orig(case, net, th_hat_b, qmax2, dt, U, 2.0 - den, b_t)  # 1 + y a^T u instead of 1 - y a^T u
    monkeypatch.setattr(Q, "_ctg_period_smw", bad)
    assert abs(oracle.evaluate(c, x, mode="smw").obj - good.obj) > 1e-6 * abs(good.obj)


# --------------------------------------------------------------------------------------------
# warm-start MLP oracle
# --------------------------------------------------------------------------------------------

def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(3)
    n_in, n_h, n_out, B = 7, 5, 3, 4
    npar = n_h * n_in + n_h + n_h * n_h + n_h + n_out * n_h + n_out
    w = rng.normal(0, 0.5, npar)
    X = rng.normal(size=(B, n_in))
    Tg = rng.normal(size=(B, n_out))
    _, _, g = mlp.forward_backward(w, X, Tg, n_in, n_h, n_out, quantize=False)
    h = 1e-6
    for i in range(npar):
        wp = w.copy(); wp[i] += h
        wm = w.copy(); wm[i] -= h
        fd = (mlp.loss_only(wp, X, Tg, n_in, n_h, n_out) - mlp.loss_only(wm, X, Tg, n_in, n_h, n_out)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), i


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    from oracle import mlp
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-8, 8, 1000), [0.0, -0.0, 1.0, 3.0e38]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(a), ref)


def test_sparse_lu_route_agrees_with_the_explicit_inverse():
    """Large grids go through a sparse LU factorization of the reduced Laplacian, small ones through
    its explicit inverse: the same solves (Eqs. Yb_solve, 2nd_lin_sys), equal to rounding on a grid
    both can take.  The explicit-inverse route is pinned by the tests above."""
    c = synth.mid()
    x = synth.random_point(c, 3)
    rd = oracle.evaluate(c, x, net=oracle.dc_network(c, sparse=False))
    rs = oracle.evaluate(c, x, net=oracle.dc_network(c, sparse=True))
    assert abs(rs.obj - rd.obj) <= 1e-11 * abs(rd.obj)
    assert np.linalg.norm(rs.grad - rd.grad) <= 1e-10 * np.linalg.norm(rd.grad)
    for k in oracle.TERM_NAMES:
        assert abs(rs.terms[k] - rd.terms[k]) <= 1e-11 * max(abs(rd.terms[k]), 1e-6 * abs(rd.obj))


# --------------------------------------------------------------------------------------------
# transformers and phase shifters (tap ratio tau, phase shift phi as variables)
# --------------------------------------------------------------------------------------------

def _tiny_xf():
    return synth.with_transformers(synth.tiny(), frac=0.3, seed=4)


@pytest.mark.parametrize("seed", [1, 3])
def test_fd_gradient_tiny_transformers_all_coordinates(seed):
    """Every coordinate, tau and phi included, against central differences of the objective."""
    c = _smooth(_tiny_xf())
    assert c.n_xf >= 4 and np.any(c.phi_max > 0)
    x = synth.random_point(c, seed)
    g = oracle.evaluate(c, x).grad
    fd = _fd(c, x, np.arange(c.n_x))
    scale = np.abs(g).max()
    assert np.max(np.abs(fd - g)) <= 1e-7 * scale, np.max(np.abs(fd - g)) / scale
    otau, ophi = c.offsets_xf()
    assert np.abs(g[otau:]).max() > 1e-3 * scale  # the new coordinates carry real gradient


@pytest.mark.parametrize("mk", [_tiny_xf, lambda: synth.with_transformers(synth.batch(per_shape=1)[0], 0.2, 5)])
def test_ctg_smw_matches_brute_force_with_phase_shifters(mk):
    """The rank-1 form with phase-shift flows (the outaged branch losing its own b_k) against
    re-solving every outaged network with its phase-shift injections."""
    c = mk()
    x = synth.random_point(c, 13)
    a = oracle.evaluate(c, x, mode="smw")
    b = oracle.evaluate(c, x, mode="brute")
    assert abs(a.obj - b.obj) <= 1e-12 * abs(b.obj)
    assert np.allclose(a.z_ctg, b.z_ctg, rtol=1e-12, atol=0)
    assert np.max(np.abs(a.grad - b.grad)) <= 1e-11 * np.abs(b.grad).max()


@pytest.mark.parametrize("tau,phi", [(1.0, 0.0), (0.93, 0.0), (1.07, 0.2), (1.0, -0.25)])
def test_two_bus_transformer_against_complex_power(tau, phi):
    """Ideal transformer 1 : tau e^{j phi}... written as the series admittance seen through the tap:
    V_f' = V_f e^{-j phi} / tau, I_fr = (y_sr (V_f' - V_o) + j b_ch/2 V_f') e^{-j phi} / tau."""
    xl, bch, rr = 0.2, 0.04, 0.05
    c = _two_bus(xl, bch, rr)
    c = dataclasses.replace(c, xf_branch=np.array([0], np.int32), tau_min=np.array([0.9]), tau_max=np.array([1.1]),
                            phi_min=np.array([-0.3]), phi_max=np.array([0.3]))
    f, o = int(c.br_from[0]), int(c.br_to[0])
    rng = np.random.default_rng(1)
    v = rng.uniform(0.9, 1.1, (1, 2))
    th = rng.normal(0, 0.3, (1, 2))
    pf, qf, pt, qt = oracle.ac_flows(c, v, th, np.array([[tau]]), np.array([[phi]]))
    Vf = v[0, f] * np.exp(1j * th[0, f])
    Vo = v[0, o] * np.exp(1j * th[0, o])
    ysr = 1.0 / (rr + 1j * xl)
    Vfp = Vf * np.exp(-1j * phi) / tau
    Ifp = ysr * (Vfp - Vo) + 1j * bch / 2 * Vfp
    It = ysr * (Vo - Vfp) + 1j * bch / 2 * Vo
    Sf = Vfp * np.conj(Ifp)  # power into the line at the ideal transformer's secondary = at the primary
    St = Vo * np.conj(It)
    assert abs(pf[0, 0] - Sf.real) < 1e-13 and abs(qf[0, 0] - Sf.imag) < 1e-13
    assert abs(pt[0, 0] - St.real) < 1e-13 and abs(qt[0, 0] - St.imag) < 1e-13


def test_phase_shifted_flows_conserve_injections():
    """DC base flows with phase shifters satisfy KCL (E^T p = pbar) and equal y (theta_f - theta_o
    - phi) on every branch (the contingency flow equation of Sec. II-E)."""
    c = _tiny_xf()
    x = synth.random_point(c, 14)
    v, th, p, q, r, tau, phi = oracle.unpack(c, x)
    net = oracle.dc_network(c)
    _, pbar = oracle.dc_injections(c, p)
    phib = Q.branch_tau_phi(c, tau, phi)[1]
    bflow = Q.phase_shift_flows(c, net, phib)
    thd, flow = oracle.dc_base_flows(c, net, pbar, bflow)
    assert np.allclose(flow @ net.E, pbar, atol=1e-12)
    dth = thd[:, c.br_from] - thd[:, c.br_to] - phib
    assert np.allclose(flow, net.y[None, :] * dth, atol=1e-12)
