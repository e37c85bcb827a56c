"""Copper-plate economic dispatch bound (Sec. III-A, Projection "Copper Plate Economic Dispatch").

TEST INFRASTRUCTURE ONLY (see qg_oracle.py).

The paper drops the network, contingencies and integrality and solves an LP.
With the quadratic generator costs of the synthetic cases the relaxation is a
convex QP; it is solved here exactly by outer approximation: each quadratic
cost a p^2 + b p is replaced by the maximum of its tangent lines, an LP is
solved with scipy's HiGHS, a tangent is added at every point where the cost is
underestimated, and the loop repeats until the underestimate is below tol.  The
LP value is a valid lower bound at every iteration.

Relaxation kept (every dropped term of Phi is >= 0 at eps = 0):
    sum_t d_t [ sum_g (a p^2 + b p + c^r r) + c^p beta max(0, L_t - sum_g p)
               + sum_z c^rz beta max(0, R_zt - sum_{g in z} r) ]
    + rho beta sum (headroom and ramp violations),      p in [pmin, pmax], r in [0, pmax].
The balance term is a lower bound of sum_i c^p |P_it| because sum_i P_it equals
load - generation + branch losses and every branch loss g |V_f - V_o|^2 is >= 0.

contingency_bound adds what the copper plate drops but the method's own model
keeps exact in the dispatch: the DC post-contingency flows of Sec. II-E are
affine in p, so their overload terms enter the LP as linear pieces.  It is a
valid lower bound of Phi at eps = 0 as well, and a tighter one wherever no
dispatch avoids every post-contingency overload.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog


def _require_plain_devices(case, what):
    """Both LPs model producers with quadratic costs only; the device models of Examples 2-4 would
    need their own relaxations, so such cases are refused rather than bounded wrongly."""
    if (np.size(case.blk_width) and np.any(np.asarray(case.blk_width) > 0)) or np.any(case.dev_cons) or case.commit:
        raise ValueError(f"{what}: bid blocks, consumers and on-status are not modelled")


def _base_lp(case):
    """Variables, bounds, linear cost and rows of the copper-plate LP (without the cost cuts).

    Variable blocks: p[T,G], r[T,G], c[T,G] (cost epigraph), s[T] (unserved), u[T,Z] (reserve
    shortfall), h[T,G] (headroom violation), ru[T-1,G], rd[T-1,G] (ramp violations)."""
    T, G, Z = case.T, case.n_gen, case.n_zone
    dt = case.dt
    beta = case.beta
    nTG = T * G
    nR = max(T - 1, 0) * G
    idx = {}
    off = 0
    for name, size in (("p", nTG), ("r", nTG), ("c", nTG), ("s", T), ("u", T * Z), ("h", nTG),
                       ("ru", nR), ("rd", nR)):
        idx[name] = off
        off += size
    nv = off
    cost = np.zeros(nv)
    cost[idx["r"]:idx["r"] + nTG] = (dt[:, None] * case.cost_r[None, :]).ravel()
    cost[idx["c"]:idx["c"] + nTG] = np.repeat(dt, G)
    cost[idx["s"]:idx["s"] + T] = dt * case.c_p * beta
    cost[idx["u"]:idx["u"] + T * Z] = np.repeat(dt, Z) * case.c_rz * beta
    cost[idx["h"]:idx["h"] + nTG] = case.rho * beta
    cost[idx["ru"]:idx["ru"] + nR] = case.rho * beta
    cost[idx["rd"]:idx["rd"] + nR] = case.rho * beta
    lb = np.zeros(nv)
    ub = np.full(nv, np.inf)
    lb[idx["p"]:idx["p"] + nTG] = np.tile(case.pmin, T)
    ub[idx["p"]:idx["p"] + nTG] = np.tile(case.pmax, T)
    ub[idx["r"]:idx["r"] + nTG] = np.tile(case.pmax, T)
    lb[idx["c"]:idx["c"] + nTG] = -np.inf

    rows, cols, vals, rhs = [], [], [], []
    nrow = 0

    def add_row(cs, vs, bound):
        nonlocal nrow
        rows.extend([nrow] * len(cs)); cols.extend(cs); vals.extend(vs); rhs.append(bound)
        nrow += 1

    L = case.load_p.sum(axis=1)
    for t in range(T):
        # L_t - sum p <= s_t   ->  -sum p - s <= -L
        add_row([idx["p"] + t * G + g for g in range(G)] + [idx["s"] + t], [-1.0] * G + [-1.0], -L[t])
        for z in range(Z):
            gz = np.nonzero(case.gen_zone == z)[0]
            add_row([idx["r"] + t * G + g for g in gz] + [idx["u"] + t * Z + z], [-1.0] * len(gz) + [-1.0],
                    -case.reserve_req[t, z])
        for g in range(G):
            k = t * G + g
            add_row([idx["p"] + k, idx["r"] + k, idx["h"] + k], [1.0, 1.0, -1.0], case.pmax[g])
            if t >= 1:
                kp = (t - 1) * G + g
                kr = (t - 1) * G + g
                lim = case.ramp[g] * dt[t]
                add_row([idx["p"] + k, idx["p"] + kp, idx["ru"] + kr], [1.0, -1.0, -1.0], lim)
                add_row([idx["p"] + kp, idx["p"] + k, idx["rd"] + kr], [1.0, -1.0, -1.0], lim)
    return idx, nv, cost, lb, ub, (rows, cols, vals, rhs, nrow)


def _initial_cuts(case, init_cuts):
    T, G = case.T, case.n_gen
    cuts = [[] for _ in range(T * G)]
    for t in range(T):
        for g in range(G):
            for p0 in np.linspace(case.pmin[g], case.pmax[g], init_cuts):
                cuts[t * G + g].append(float(p0))
    return cuts


def _add_cuts(case, idx, cuts, rows, cols, vals, rhs, nrow):
    """Tangent cuts c >= a (2 p0 p - p0^2) + b p, i.e. (2 a p0 + b) p - c <= a p0^2."""
    G = case.n_gen
    a, b = case.cost_a, case.cost_b
    for k, pts in enumerate(cuts):
        g = k % G
        for p0 in pts:
            rows.extend([nrow, nrow]); cols.extend([idx["p"] + k, idx["c"] + k])
            vals.extend([2 * a[g] * p0 + b[g], -1.0]); rhs.append(a[g] * p0 * p0); nrow += 1
    return nrow


def _cost_gap(case, idx, xs):
    """Underestimate of the quadratic cost by the cut epigraph at the LP solution, per (t, g)."""
    nTG = case.T * case.n_gen
    G = case.n_gen
    p = xs[idx["p"]:idx["p"] + nTG]
    c = xs[idx["c"]:idx["c"] + nTG]
    g = np.arange(nTG) % G
    return case.cost_a[g] * p * p + case.cost_b[g] * p - c, p


def copper_plate(case, tol: float = 1e-9, max_rounds: int = 60, init_cuts: int = 6):
    """Returns (bound, p [T, G], r [T, G])."""
    _require_plain_devices(case, "copper_plate")
    T, G = case.T, case.n_gen
    nTG = T * G
    idx, nv, cost, lb, ub, base_rows = _base_lp(case)
    cuts = _initial_cuts(case, init_cuts)
    best = None
    for _round in range(max_rounds):
        rows, cols, vals, rhs = (list(base_rows[0]), list(base_rows[1]), list(base_rows[2]), list(base_rows[3]))
        nrow = _add_cuts(case, idx, cuts, rows, cols, vals, rhs, base_rows[4])
        A = sp.csr_matrix((vals, (rows, cols)), shape=(nrow, nv))
        res = linprog(cost, A_ub=A, b_ub=np.array(rhs), bounds=list(zip(lb, ub)), method="highs")
        if res.status != 0:
            raise RuntimeError(f"copper-plate LP failed: {res.message}")
        xs = res.x
        gap, p = _cost_gap(case, idx, xs)
        best = (res.fun, p.reshape(T, G).copy(), xs[idx["r"]:idx["r"] + nTG].reshape(T, G).copy())
        total = abs(res.fun) + 1.0
        if gap.max() * T * G <= tol * total:
            break
        for k in np.nonzero(gap > 0.1 * tol * total / (T * G))[0]:
            cuts[k].append(float(p[k]))
    return best


def contingency_flow_maps(case, net=None):
    """The post-contingency DC flows of Sec. II-E as affine maps of the dispatch.

    With the uniform slack, the base flows of period t are f_t = J p_t + f0_t (J [M, G]: flow per
    unit of each device's output, the imbalance spread over all buses; f0_t [M]: the flows of the
    load alone), and the rank-1 correction (Eq. rank_correct, in flow space) gives the flow on
    branch m after outage k as F_t[m, k] = f_t[m] + Lo[m, k] f_t[ctg_k], with
    Lo[m, k] = y_m a_m^T u_k / (1 - y_k a_k^T u_k), u_k = Yhat^-1 a_k, and Lo = 0 on each outage's
    own branch.  Returns (J, f0 [T, M], Lo [M, K])."""
    from . import qg_oracle as Q
    net = Q.dc_network(case) if net is None else net
    G, n = case.n_gen, case.n_bus
    U, den = Q.outage_columns(case, net)
    Eh = net.E[:, net.keep]
    y = net.y
    Lo = y[:, None] * np.asarray(Eh @ U) / den[None, :]
    Lo[case.ctg, np.arange(len(case.ctg))] = 0.0
    A = np.zeros((n, G))
    A[case.gen_bus, np.arange(G)] = Q.device_sign(case)
    Ab = A - A.mean(axis=0, keepdims=True)
    J = y[:, None] * np.asarray(Eh @ net.solve(Ab[net.keep]))
    _, f0 = Q.dc_base_flows(case, net, Q.dc_injections(case, np.zeros((case.T, G)))[1])
    return J, f0, Lo


def contingency_bound(case, tol: float = 1e-9, max_rounds: int = 80, init_cuts: int = 6, net=None):
    """A lower bound of Phi at eps = 0 that keeps the DC contingency overloads.

    The copper-plate relaxation above plus, for a set S of (period, monitored branch, outage)
    triples, the term d_t c^s beta max(0, |F_t[m, k]| - s^ctg_m) with F the affine post-contingency
    flow of contingency_flow_maps.  Each such term is a lower bound of the triple's share of z_tk
    (s = sqrt(F^2 + qmax^2) >= |F|, and the soft-ReLU at eps = 0 is the plain ReLU), and every
    triple left out of S contributes >= 0, so the LP value is a valid lower bound for any S.  S
    starts with the triples overloaded at the copper-plate dispatch and grows by the ones overloaded
    at each LP solution, together with tangent cuts of the cost, until the relaxed objective at the
    LP solution (true cost, every triple) exceeds the LP value by at most tol of it: the returned
    value is then within that margin of the relaxation's minimum.  The model is exact in p: F is
    the method's own DC contingency flow.
    Returns (bound, p [T, G], r [T, G], number of triples in S)."""
    _require_plain_devices(case, "contingency_bound")
    if len(case.xf_branch):
        raise ValueError("contingency_bound: phase shifters add flow terms the maps leave out")
    T, G = case.T, case.n_gen
    nTG = T * G
    ctg = np.asarray(case.ctg)
    K = len(ctg)
    if K == 0:
        b, p, r = copper_plate(case, tol, max_rounds, init_cuts)
        return b, p, r, 0
    J, f0, Lo = contingency_flow_maps(case, net)
    smax = case.s_max_ctg
    w_t = case.dt * case.c_s * case.beta
    idx, nv, cost, lb, ub, base_rows = _base_lp(case)
    cuts = _initial_cuts(case, init_cuts)

    def overloads(p):
        f = p @ J.T + f0                                        # [T, M]
        F = f[:, :, None] + Lo[None, :, :] * f[:, ctg][:, None, :]
        v = np.abs(F) - smax[None, :, None]
        v[:, ctg, np.arange(K)] = -np.inf                      # the outaged branch is not monitored
        return v

    _, p_cp, _ = copper_plate(case, tol, max_rounds, init_cuts)
    tS, mS, kS = np.nonzero(overloads(p_cp) > 0)
    best = None
    for _round in range(max_rounds):
        nS = len(tS)
        rows, cols, vals, rhs = (list(base_rows[0]), list(base_rows[1]), list(base_rows[2]), list(base_rows[3]))
        nrow = _add_cuts(case, idx, cuts, rows, cols, vals, rhs, base_rows[4])
        # |a . p_t + b| - s_m <= o_j as two rows per triple: (+-a) . p_t - o_j <= s_m -+ b
        a = J[mS] + Lo[mS, kS][:, None] * J[ctg[kS]]             # [nS, G]
        b0 = f0[tS, mS] + Lo[mS, kS] * f0[tS, ctg[kS]]
        pc = idx["p"] + tS[:, None] * G + np.arange(G)[None, :]
        oc = nv + np.arange(nS)
        R = [np.array(rows, dtype=np.int64)]
        C = [np.array(cols, dtype=np.int64)]
        V = [np.array(vals)]
        rh = [np.array(rhs)]
        for sgn, r0 in ((1.0, nrow), (-1.0, nrow + nS)):
            rr = r0 + np.arange(nS)
            R += [np.repeat(rr, G), rr]
            C += [pc.ravel(), oc]
            V += [(sgn * a).ravel(), -np.ones(nS)]
            rh.append(smax[mS] - sgn * b0)
        A = sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(nrow + 2 * nS, nv + nS))
        cost_all = np.concatenate([cost, w_t[tS]])
        bounds = list(zip(lb, ub)) + [(0.0, None)] * nS
        res = linprog(cost_all, A_ub=A, b_ub=np.concatenate(rh), bounds=bounds, method="highs")
        if res.status != 0:
            raise RuntimeError(f"contingency bound LP failed: {res.message}")
        xs = res.x
        gap, p = _cost_gap(case, idx, xs)
        best = (res.fun, p.reshape(T, G).copy(), xs[idx["r"]:idx["r"] + nTG].reshape(T, G).copy(), nS)
        total = abs(res.fun) + 1.0
        v = overloads(p.reshape(T, G))
        have = np.zeros(v.shape, bool)
        have[tS, mS, kS] = True
        tN, mN, kN = np.nonzero((v > 0) & ~have)
        # relaxed objective at the solution minus the LP value: cost underestimate + overloads not in S
        excess = np.dot(np.repeat(case.dt, G), gap) + (w_t[tN] * v[tN, mN, kN]).sum()
        if excess <= tol * total:
            break
        for k in np.nonzero(gap > 0.1 * tol * total / (T * G))[0]:
            cuts[k].append(float(p[k]))
        tS, mS, kS = np.concatenate([tS, tN]), np.concatenate([mS, mN]), np.concatenate([kS, kN])
    return best


def lambda_dispatch(case, tol: float = 1e-12):
    """Single-period copper-plate optimum without reserve or ramp terms, per period:
    p_g = clip((lam - b_g) / (2 a_g), pmin_g, pmax_g) with lam chosen by bisection so that
    sum_g p_g equals the period's load (the KKT conditions of the quadratic dispatch)."""
    T = case.T
    out = np.zeros((T, case.n_gen))
    a, b = case.cost_a, case.cost_b
    for t in range(T):
        L = case.load_p[t].sum()
        lo, hi = 0.0, float(b.max() + 2 * (a * case.pmax).max()) + 1.0
        for _ in range(200):
            lam = 0.5 * (lo + hi)
            s = np.clip((lam - b) / (2 * a), case.pmin, case.pmax).sum()
            if s < L:
                lo = lam
            else:
                hi = lam
            if hi - lo < tol:
                break
        out[t] = np.clip((0.5 * (lo + hi) - b) / (2 * a), case.pmin, case.pmax)
    return out
