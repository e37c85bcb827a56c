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
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog


def copper_plate(case, tol: float = 1e-9, max_rounds: int = 60, init_cuts: int = 6):
    """Returns (bound, p [T, G], r [T, G])."""
    T, G, Z = case.T, case.n_gen, case.n_zone
    dt = case.dt
    beta = case.beta
    a, b = case.cost_a, case.cost_b
    # variable blocks: p[T,G], r[T,G], c[T,G] (cost epigraph), s[T] (unserved), u[T,Z] (reserve
    # shortfall), h[T,G] (headroom violation), ru[T-1,G], rd[T-1,G] (ramp violations)
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
    base_rows = (list(rows), list(cols), list(vals), list(rhs), nrow)

    # tangent cuts: c >= a (2 p0 p - p0^2) + b p   ->   (2 a p0 + b) p - c <= a p0^2
    cuts = [[] for _ in range(nTG)]
    for t in range(T):
        for g in range(G):
            for p0 in np.linspace(case.pmin[g], case.pmax[g], init_cuts):
                cuts[t * G + g].append(float(p0))

    best = None
    for _round in range(max_rounds):
        rows, cols, vals, rhs, nrow = (list(base_rows[0]), list(base_rows[1]), list(base_rows[2]),
                                       list(base_rows[3]), base_rows[4])
        for k in range(nTG):
            g = k % G
            for p0 in cuts[k]:
                rows.extend([nrow, nrow]); cols.extend([idx["p"] + k, idx["c"] + k])
                vals.extend([2 * a[g] * p0 + b[g], -1.0]); rhs.append(a[g] * p0 * p0); nrow += 1
        A = sp.csr_matrix((vals, (rows, cols)), shape=(nrow, nv))
        res = linprog(cost, A_ub=A, b_ub=np.array(rhs), bounds=list(zip(lb, ub)), method="highs")
        if res.status != 0:
            raise RuntimeError(f"copper-plate LP failed: {res.message}")
        xs = res.x
        p = xs[idx["p"]:idx["p"] + nTG]
        c = xs[idx["c"]:idx["c"] + nTG]
        true_c = a[np.arange(nTG) % G] * p * p + b[np.arange(nTG) % G] * p
        gap = true_c - c
        best = (res.fun, p.reshape(T, G).copy(), xs[idx["r"]:idx["r"] + nTG].reshape(T, G).copy())
        total = abs(res.fun) + 1.0
        if gap.max() * T * G <= tol * total:
            break
        for k in np.nonzero(gap > 0.1 * tol * total / (T * G))[0]:
            cuts[k].append(float(p[k]))
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
