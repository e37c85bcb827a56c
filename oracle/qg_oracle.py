"""FP64 CPU oracle of the QuasiGrad penalized objective and its gradient.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module; the library's product path never does.
It shares no code with the CUDA path (different layout, different loop order:
contingencies are evaluated per outage in angle space exactly as Sec. II-E
describes, not through a flow-space LODF block).

What it computes (plain definitions, numpy FP64):

* AC branch flows of the pi model (Sec. II-F line-flow example fixes the sign
  convention: d p_fr / d v_to = (-g cos(delta) - b sin(delta)) v_fr / tau), with
  tau = 1, phi = 0 and no per-end shunt conductance/susceptance.
* Bus P/Q mismatch (Example 4, consumption positive) and the soft-abs balance
  penalty (Sec. II-C footnote; scaled by beta as in the homotopy paragraph of
  Sec. II-F).
* Thermal penalty on the worse branch end (Example 1) with the soft-ReLU.
* Generator cost, reserve cost, zonal reserve shortfall, headroom and ramp
  penalties (the penalized linear constraints rho*sigma_s(Ax) of Eq. nlp_updated,
  applied to violations).
* Contingency DC flows (Sec. II-E): base solve of the reduced Laplacian with
  uniform slack, SMW rank-1 correction per outage (Eq. rank_correct), the
  directional overload penalty (Eqs. sfr_pen-zctg), the adjoint solve
  (Eq. 2nd_lin_sys) and the slack correction (Eq. correction).
  ``mode="brute"`` instead deletes the outaged branch and re-solves the
  contingency Laplacian directly.
  Linear solves with the reduced Laplacian use its explicit inverse for small
  grids and a sparse LU factorization (scipy SuperLU) above SPARSE_N buses;
  both are the same solve of Eqs. Yb_solve and 2nd_lin_sys.

Readings taken where the paper is silent or ambiguous are listed in the
design notes; the ones that change arithmetic are repeated at their use below.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SPARSE_N = 4096  # grids above this many buses are solved through a sparse factorization


# ------------------------------------------------------------------------------------------
# smooth penalties (Sec. II-C footnote)
# ------------------------------------------------------------------------------------------

def soft_abs(x, eps):
    """|x|_s = sqrt(x^2 + eps^2)."""
    return np.sqrt(x * x + eps * eps)


def soft_abs_grad(x, eps):
    s = np.sqrt(x * x + eps * eps)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(s > 0, x / np.where(s > 0, s, 1.0), 0.0)


def soft_relu(x, eps):
    """sigma_s(x) = sqrt(max(x, 0)^2 + eps^2)."""
    m = np.maximum(x, 0.0)
    return np.sqrt(m * m + eps * eps)


def soft_relu_grad(x, eps):
    m = np.maximum(x, 0.0)
    s = np.sqrt(m * m + eps * eps)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(s > 0, m / np.where(s > 0, s, 1.0), 0.0)


# ------------------------------------------------------------------------------------------
# variable layout
# ------------------------------------------------------------------------------------------

def _n_xf(case):
    return int(getattr(case, "n_xf", 0))


def unpack(case, x):
    """x = [v (T x n) | theta (T x n) | p (T x G) | q (T x G) | r (T x G) | tau (T x X) | phi (T x X)],
    period-major rows; X transformers (tau, phi blocks absent when X = 0)."""
    T, n, G, X = case.T, case.n_bus, case.n_gen, _n_xf(case)
    x = np.asarray(x, dtype=np.float64)
    o = 0
    v = x[o:o + T * n].reshape(T, n); o += T * n
    th = x[o:o + T * n].reshape(T, n); o += T * n
    p = x[o:o + T * G].reshape(T, G); o += T * G
    q = x[o:o + T * G].reshape(T, G); o += T * G
    r = x[o:o + T * G].reshape(T, G); o += T * G
    if X == 0:
        return v, th, p, q, r
    tau = x[o:o + T * X].reshape(T, X); o += T * X
    phi = x[o:o + T * X].reshape(T, X)
    return v, th, p, q, r, tau, phi


def unpack_u(case, x):
    """The on-status block u (T x G) that follows phi when the case has commitment, else None."""
    if not getattr(case, "commit", False):
        return None
    T, G = case.T, case.n_gen
    o = T * (2 * case.n_bus + 3 * G + 2 * _n_xf(case))
    return np.asarray(x, dtype=np.float64)[o:o + T * G].reshape(T, G)


def pack(v, th, p, q, r, tau=None, phi=None, u=None):
    parts = [np.ravel(v), np.ravel(th), np.ravel(p), np.ravel(q), np.ravel(r)]
    if tau is not None:
        parts += [np.ravel(tau), np.ravel(phi)]
    if u is not None:
        parts.append(np.ravel(u))
    return np.concatenate(parts)


def device_sign(case):
    """+1 for producers, -1 for consumers: the sign with which a device's p, q enter as supply."""
    cons = getattr(case, "dev_cons", None)
    if cons is None or len(cons) == 0:
        return np.ones(case.n_gen)
    return np.where(np.asarray(cons, bool), -1.0, 1.0)


def box(case):
    """Clip box B of Alg. 3 (clip step): v in [vmin, vmax], theta_ref = 0, other theta free,
    p in [pmin, pmax], q in [qmin, qmax], r in [0, pmax] (consumers: r = 0), tau and phi in their
    ranges.  With commitment the limits scaled by u become penalized constraints, and the box keeps
    p in [0, pmax], q in [min(qmin, 0), max(qmax, 0)] and u in [0, 1]."""
    T, n, G, X = case.T, case.n_bus, case.n_gen, _n_xf(case)
    commit = bool(getattr(case, "commit", False))
    lo_th = np.full((T, n), -np.inf)
    hi_th = np.full((T, n), np.inf)
    lo_th[:, case.ref_bus] = 0.0
    hi_th[:, case.ref_bus] = 0.0
    xl = (np.tile(case.tau_min, (T, 1)), np.tile(case.phi_min, (T, 1))) if X else (None, None)
    xh = (np.tile(case.tau_max, (T, 1)), np.tile(case.phi_max, (T, 1))) if X else (None, None)
    plo = np.zeros(G) if commit else case.pmin
    qlo = np.minimum(case.qmin, 0.0) if commit else case.qmin
    qhi = np.maximum(case.qmax, 0.0) if commit else case.qmax
    rhi = np.where(device_sign(case) < 0, 0.0, case.pmax)
    ul, uh = (np.zeros((T, G)), np.ones((T, G))) if commit else (None, None)
    lo = pack(np.tile(case.vmin, (T, 1)), lo_th, np.tile(plo, (T, 1)), np.tile(qlo, (T, 1)),
              np.zeros((T, G)), *xl, u=ul)
    hi = pack(np.tile(case.vmax, (T, 1)), hi_th, np.tile(case.pmax, (T, 1)), np.tile(qhi, (T, 1)),
              np.tile(rhi, (T, 1)), *xh, u=uh)
    return lo, hi


def branch_tau_phi(case, tau, phi):
    """(T, M) tap ratio and phase shift of every branch: the transformer variables on transformer
    branches, tau = 1 and phi = 0 on lines."""
    T, M = case.T, case.n_branch
    tb = np.ones((T, M))
    pb = np.zeros((T, M))
    if tau is not None:
        tb[:, case.xf_branch] = tau
        pb[:, case.xf_branch] = phi
    return tb, pb


# ------------------------------------------------------------------------------------------
# AC network (pi model)
# ------------------------------------------------------------------------------------------

def series_admittance(case):
    """g_sr + j b_sr = 1 / (r + j x)."""
    den = case.br_r ** 2 + case.br_x ** 2
    return case.br_r / den, -case.br_x / den


def ac_flows(case, v, th, tau=None, phi=None):
    """Pi-model flows at both ends of every branch, shape (T, M) each; an ideal transformer of tap
    ratio tau and phase shift phi sits at the "fr" end (tau = 1, phi = 0 on lines):

    p_fr = g v_f^2 / tau^2 + (-g cos d - b sin d) v_f v_o / tau
    q_fr = -(b + b_ch/2) v_f^2 / tau^2 + (b cos d - g sin d) v_f v_o / tau
    p_to = g v_o^2 + (-g cos d + b sin d) v_f v_o / tau
    q_to = -(b + b_ch/2) v_o^2 + (b cos d + g sin d) v_f v_o / tau,   d = theta_f - theta_o - phi.
    """
    g, b = series_admittance(case)
    bch = case.br_b
    f, o = case.br_from, case.br_to
    tb, pb = branch_tau_phi(case, tau, phi)
    vf, vo = v[:, f], v[:, o]
    d = th[:, f] - th[:, o] - pb
    c, s = np.cos(d), np.sin(d)
    vv = vf * vo / tb
    vf2 = vf ** 2 / tb ** 2
    pf = g * vf2 + (-g * c - b * s) * vv
    qf = -(b + bch / 2) * vf2 + (b * c - g * s) * vv
    pt = g * vo ** 2 + (-g * c + b * s) * vv
    qt = -(b + bch / 2) * vo ** 2 + (b * c + g * s) * vv
    return pf, qf, pt, qt


def ac_flow_partials(case, v, th, tau=None, phi=None):
    """Partial derivatives of (pf, qf, pt, qt) with respect to (v_f, v_o, delta, tau);
    d/dtheta_f = d/ddelta, d/dtheta_o = d/dphi = -d/ddelta."""
    g, b = series_admittance(case)
    bch = case.br_b
    f, o = case.br_from, case.br_to
    tb, pb = branch_tau_phi(case, tau, phi)
    vf, vo = v[:, f], v[:, o]
    d = th[:, f] - th[:, o] - pb
    c, s = np.cos(d), np.sin(d)
    vv = vf * vo / tb
    out = {
        "pf": (2 * g * vf / tb ** 2 + (-g * c - b * s) * vo / tb, (-g * c - b * s) * vf / tb, (g * s - b * c) * vv,
               -2 * g * vf ** 2 / tb ** 3 - (-g * c - b * s) * vv / tb),
        "qf": (-2 * (b + bch / 2) * vf / tb ** 2 + (b * c - g * s) * vo / tb, (b * c - g * s) * vf / tb,
               (-b * s - g * c) * vv, 2 * (b + bch / 2) * vf ** 2 / tb ** 3 - (b * c - g * s) * vv / tb),
        "pt": ((-g * c + b * s) * vo / tb, 2 * g * vo + (-g * c + b * s) * vf / tb, (g * s + b * c) * vv,
               -(-g * c + b * s) * vv / tb),
        "qt": ((b * c + g * s) * vo / tb, -2 * (b + bch / 2) * vo + (b * c + g * s) * vf / tb, (-b * s + g * c) * vv,
               -(b * c + g * s) * vv / tb),
    }
    return out


def energy_cost(case, p):
    """(z, dz/dp), each (T, G): the energy cost (producers) or value (consumers) per hour before d_t.
    A device with bid blocks (Example 3): z = sum_l c_l max(min(p - P_{l-1}, w_l), 0) with
    P_{l-1} = w_1 + ... + w_{l-1}; its derivative is taken from the right (the price of the block
    that p is entering: the one with 0 <= p - P_{l-1} < w_l, and 0 past the last block).  Devices
    without blocks (all widths 0): z = a p^2 + b p."""
    z = case.cost_a * p * p + case.cost_b * p
    dz = 2 * case.cost_a * p + case.cost_b
    W = getattr(case, "blk_width", None)
    if W is None or W.size == 0:
        return z, dz
    C = case.blk_price
    has = W.sum(axis=1) > 0
    lo = np.zeros_like(W)
    for l in range(1, W.shape[1]):
        lo[:, l] = lo[:, l - 1] + W[:, l - 1]
    zb = np.zeros_like(p)
    db = np.zeros_like(p)
    for l in range(W.shape[1]):
        d = p - lo[None, :, l]
        zb += C[None, :, l] * np.maximum(np.minimum(d, W[None, :, l]), 0.0)
        db += np.where((d >= 0) & (d < W[None, :, l]), C[None, :, l], 0.0)
    return np.where(has[None, :], zb, z), np.where(has[None, :], db, dz)


def bus_mismatch(case, pf, qf, pt, qt, p, q):
    """Example 4: P_it = sum(loads) + sum(consumers) + sum(fr flows) + sum(to flows) - sum(producers),
    same for Q (the fixed loads are consumption that has no variable)."""
    f, o = case.br_from, case.br_to
    P = case.load_p.copy()
    Q = case.load_q.copy()
    np.add.at(P.T, f, pf.T)
    np.add.at(P.T, o, pt.T)
    np.add.at(Q.T, f, qf.T)
    np.add.at(Q.T, o, qt.T)
    sg = device_sign(case)
    np.subtract.at(P.T, case.gen_bus, (sg * p).T)
    np.subtract.at(Q.T, case.gen_bus, (sg * q).T)
    return P, Q


# ------------------------------------------------------------------------------------------
# DC network (Sec. II-E)
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass
class DCNet:
    y: np.ndarray        # [M] branch susceptance -b_sr = x / (r^2 + x^2)
    E: object            # [M, n] signed incidence (+1 at from, -1 at to); scipy CSR when sparse
    keep: np.ndarray     # [n-1] bus ids with the reference bus removed
    Yhat: object         # [n-1, n-1] reduced Laplacian  E_hat^T Y_x E_hat
    Yinv: Optional[np.ndarray] = None  # its inverse (explicit, small cases)
    lu: object = None    # its sparse LU factorization (large cases)
    U: Optional[np.ndarray] = None     # cached u_k = Yhat^-1 a_k for the outage list ctg_of_U
    den: Optional[np.ndarray] = None
    ctg_of_U: Optional[np.ndarray] = None

    @property
    def sparse(self) -> bool:
        return self.lu is not None

    def solve(self, B):
        """Yhat^-1 B for a dense right-hand side (vector or matrix)."""
        return self.Yinv @ B if self.lu is None else self.lu.solve(np.asarray(B, dtype=np.float64))


def dc_network(case, sparse: Optional[bool] = None) -> DCNet:
    """Reading: Y_x holds -b_sr = x / (r^2 + x^2), consistent with p = -b_sr (theta_i - theta_i')."""
    n, M = case.n_bus, case.n_branch
    y = case.br_x / (case.br_r ** 2 + case.br_x ** 2)
    keep = np.array([i for i in range(n) if i != case.ref_bus])
    if sparse is None:
        sparse = n > SPARSE_N
    if sparse:
        E = sp.csr_matrix((np.r_[np.ones(M), -np.ones(M)],
                           (np.r_[np.arange(M), np.arange(M)], np.r_[case.br_from, case.br_to])), shape=(M, n))
        Eh = E[:, keep]
        Yhat = (Eh.T @ sp.diags(y) @ Eh).tocsc()
        return DCNet(y=y, E=E, keep=keep, Yhat=Yhat, lu=spla.splu(Yhat, permc_spec="MMD_AT_PLUS_A"))
    E = np.zeros((M, n))
    E[np.arange(M), case.br_from] += 1.0
    E[np.arange(M), case.br_to] -= 1.0
    Eh = E[:, keep]
    Yhat = Eh.T @ (y[:, None] * Eh)
    return DCNet(y=y, E=E, keep=keep, Yhat=Yhat, Yinv=np.linalg.inv(Yhat))


def _kdot(Ek, H):
    """[K] column-wise a_k^T H[:, k] for the rows a_k of Ek (dense or sparse)."""
    if sp.issparse(Ek):
        return np.asarray(Ek.multiply(H.T).sum(axis=1)).ravel()
    return np.einsum("kj,jk->k", Ek, H)


def outage_columns(case, net: DCNet):
    """u_k = Yhat^-1 a_k (a_k the reduced incidence row of outaged branch k) and the SMW
    denominators 1 - y_k a_k^T u_k (reading: Yhat_k = Yhat - y_k a_k a_k^T); cached on net."""
    if net.U is not None and np.array_equal(net.ctg_of_U, case.ctg):
        return net.U, net.den
    Eh = net.E[:, net.keep]
    Ak = Eh[case.ctg]
    U = net.solve(Ak.T.toarray() if net.sparse else Ak.T)
    den = 1.0 - net.y[case.ctg] * _kdot(Ak, U)
    net.U, net.den, net.ctg_of_U = U, den, np.array(case.ctg)
    return U, den


def dc_injections(case, p):
    """p_inj = producers' output - consumers' draw at the bus - load, then the uniform slack:
    every bus takes 1/n of the imbalance (Sec. II-E slack paragraph)."""
    inj = -case.load_p.copy()
    np.add.at(inj.T, case.gen_bus, (device_sign(case) * p).T)
    pbar = inj - inj.mean(axis=1, keepdims=True)
    return inj, pbar


def phase_shift_flows(case, net: DCNet, phi_b):
    """b_jt = b^sr_j phi_jt = -y_j phi_jt (Sec. II-E contingency flow equation), (T, M); 0 on lines."""
    return -net.y[None, :] * phi_b


def dc_base_flows(case, net: DCNet, pbar, bflow=None):
    """Eq. Yb_solve / p_flow: theta_hat = Yhat^-1 (pbar_hat - E_hat^T b_t).  Reading: the monitored
    flow is the physical one of the contingency flow equation, p = Y_x E_hat theta_hat + b_t (Eq.
    p_flow writes the first term only; with b_t = 0 they agree).  Returns theta (T, n) with
    theta_ref = 0 and p (T, M)."""
    rhs = pbar.copy()
    if bflow is not None:
        rhs -= (bflow @ net.E) if not net.sparse else (net.E.T @ bflow.T).T
    if net.sparse:
        th_hat = net.solve(rhs[:, net.keep].T).T
    else:
        th_hat = np.linalg.solve(net.Yhat, rhs[:, net.keep].T).T
    th = np.zeros_like(pbar)
    th[:, net.keep] = th_hat
    f = (net.E @ th.T).T * net.y[None, :] if net.sparse else (th @ net.E.T) * net.y[None, :]
    if bflow is not None:
        f = f + bflow
    return th, f


# ------------------------------------------------------------------------------------------
# contingency penalty and its gradient (Sec. II-E, Alg. 2 with every outage and zeta = 0)
# ------------------------------------------------------------------------------------------

def _ctg_period_smw(case, net: DCNet, th_hat_b, qmax2, dt, U, den, b_t=None):
    """One period, all outages, via the paper's rank-1 correction in angle space.

    th_hat_b : [n-1] base-case reduced angles (Eq. Y_base).
    U        : [n-1, K] u_k = Yhat^-1 a_k with a_k the reduced incidence row of branch k.
    den      : [K] 1 - y_k a_k^T u_k  (the SMW denominator; reading: Yhat_k = Yhat - y_k a_k a_k^T).
    b_t      : [M] phase-shift flows of the period (None: no phase shifters).  An outaged branch
               loses its own b_k with u_on = 0, so c_tk = c_t + a_k b_k and, by SMW,
               theta_tk = theta_tb + u_k (f_k + b_k) / den_k.
    Returns (z_tk [K], grad wrt p_inj [n] summed over k, dz/dqmax2 [M] summed over k,
    grad wrt b_t [M] summed over k).
    """
    K = case.K
    ks = case.ctg
    Eh = net.E[:, net.keep]
    y = net.y
    bt = np.zeros(case.n_branch) if b_t is None else b_t
    fk = y[ks] * (Eh[ks] @ th_hat_b)                        # base angle flow on each outaged branch
    TH = th_hat_b[:, None] + U * ((fk + bt[ks]) / den)[None, :]  # Eq. rank_correct, one column per k
    P = y[:, None] * (Eh @ TH) + bt[:, None]                 # Eq. p_flow plus b_t, [M, K]
    P[ks, np.arange(K)] = 0.0                                # outaged branch carries nothing
    s = np.sqrt(P * P + qmax2[:, None])
    u = s - case.s_max_ctg[:, None]
    w = dt * case.c_s * case.beta
    pen = w * soft_relu(u, case.eps)
    pen[ks, np.arange(K)] = 0.0                              # the outaged branch is not monitored
    z = pen.sum(axis=0)
    dsig = w * soft_relu_grad(u, case.eps)
    dsig[ks, np.arange(K)] = 0.0
    with np.errstate(invalid="ignore", divide="ignore"):
        inv_s = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    D = dsig * P * inv_s                                     # d_k = dz_tk / dp_tk, column per k
    gq2 = (dsig * 0.5 * inv_s).sum(axis=1)                   # dz / d(qmax^2), summed over k
    # Eq. 2nd_lin_sys: eta_k = Yhat_k^-1 E_hat^T Y_x,k d_k, with Yhat_k^-1 applied by SMW
    W = Eh.T @ (y[:, None] * D)                              # [n-1, K]
    H = net.solve(W)
    H = H + U * ((y[ks] * _kdot(Eh[ks], H)) / den)[None, :]
    eta = np.zeros((case.n_bus, K))
    eta[net.keep] = H
    gin = (eta - eta.mean(axis=0, keepdims=True)).sum(axis=1)  # Eq. correction, summed over k
    GB = D - Eh @ H                                          # Eq. 2nd_lin_sys_phase plus the direct b term
    GB[ks, np.arange(K)] = 0.0                               # b_k does not enter contingency k
    return z, gin, gq2, GB.sum(axis=1)


def _ctg_period_brute(case, net: DCNet, pbar_t, qmax2, dt, b_t=None):
    """One period, every outage re-solved on the outaged Laplacian (no SMW); the outaged branch
    also loses its phase-shift flow."""
    if net.sparse:
        raise ValueError("brute mode takes small (dense) grids only")
    K = case.K
    Eh = net.E[:, net.keep]
    y = net.y
    n = case.n_bus
    z = np.zeros(K)
    gin = np.zeros(n)
    gq2 = np.zeros(case.n_branch)
    gb = np.zeros(case.n_branch)
    bt = np.zeros(case.n_branch) if b_t is None else b_t
    w = dt * case.c_s * case.beta
    for kk, k in enumerate(case.ctg):
        yk = y.copy()
        yk[k] = 0.0
        bk = bt.copy()
        bk[k] = 0.0
        Yk = Eh.T @ (yk[:, None] * Eh)
        thk = np.linalg.solve(Yk, pbar_t[net.keep] - Eh.T @ bk)
        P = yk * (Eh @ thk) + bk
        s = np.sqrt(P * P + qmax2)
        u = s - case.s_max_ctg
        pen = w * soft_relu(u, case.eps)
        pen[k] = 0.0
        z[kk] = pen.sum()
        dsig = w * soft_relu_grad(u, case.eps)
        dsig[k] = 0.0
        inv_s = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
        d = dsig * P * inv_s
        gq2 += dsig * 0.5 * inv_s
        eta_h = np.linalg.solve(Yk, Eh.T @ (yk * d))
        eta = np.zeros(n)
        eta[net.keep] = eta_h
        gin += eta - eta.mean()
        gbk = d - Eh @ eta_h
        gbk[k] = 0.0
        gb += gbk
    return z, gin, gq2, gb


# ------------------------------------------------------------------------------------------
# the full objective and gradient
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Result:
    obj: float
    grad: Optional[np.ndarray]
    terms: dict
    z_ctg: Optional[np.ndarray] = None  # [T, K]
    g_inj: Optional[np.ndarray] = None  # [T, n] gradient of the contingency term wrt p_inj


TERM_NAMES = ("cost", "zp", "zq", "zs", "zrz", "zhead", "zramp", "zctg")


def evaluate(case, x, want_grad: bool = True, mode: str = "smw", eps: Optional[float] = None,
             periods: Optional[Sequence[int]] = None, net: Optional[DCNet] = None) -> Result:
    """Phi(x) and its gradient.

    mode: "smw" (rank-1 corrections, Eq. rank_correct) or "brute" (re-solve each outage).
    eps : override the soft-abs / soft-ReLU epsilon (eps = 0 gives the hard abs/ReLU used
          to score a point).
    periods: restrict the contingency term to these periods (sampling at large sizes);
          other terms always cover every period.
    net : the case's DC network (dc_network), to reuse its factorization across calls.
    """
    if eps is not None and eps != case.eps:
        case = dataclasses.replace(case, eps=eps)
    T, n, G, X = case.T, case.n_bus, case.n_gen, _n_xf(case)
    eps_ = case.eps
    beta = case.beta
    dt = case.dt
    if X:
        v, th, p, q, r, tau, phi = unpack(case, x)
    else:
        v, th, p, q, r = unpack(case, x)
        tau = phi = None
    gv = np.zeros((T, n)); gth = np.zeros((T, n)); gp = np.zeros((T, G)); gq = np.zeros((T, G))
    gr = np.zeros((T, G))
    terms = {k: 0.0 for k in TERM_NAMES}
    sg = device_sign(case)
    uo = unpack_u(case, x)
    gu = None if uo is None else np.zeros((T, G))

    # --- device energy cost / value (Example 3; a consumer's value enters with a minus sign, so that
    #     minimizing the objective maximizes the market surplus) and reserve cost
    zen, dzen = energy_cost(case, p)
    terms["cost"] = float((dt[:, None] * (sg * zen + case.cost_r * r)).sum())
    gp += dt[:, None] * sg * dzen
    gr += dt[:, None] * case.cost_r

    # --- on/off status (Example 2): on cost d_t c_on u, startup c_su max(u_t - u_{t-1}, 0) and shutdown
    #     c_sd max(u_{t-1} - u_t, 0), with u_init before period 0 (derivative of max(., 0) at 0 taken as 0)
    if uo is not None:
        du = uo - np.vstack([case.u_init[None, :], uo[:-1]])
        terms["cost"] += float((dt[:, None] * case.c_on * uo + case.c_su * np.maximum(du, 0.0)
                                + case.c_sd * np.maximum(-du, 0.0)).sum())
        ddu = np.where(du > 0, case.c_su, 0.0) - np.where(du < 0, case.c_sd, 0.0)
        gu += dt[:, None] * case.c_on + ddu
        gu[:-1] -= ddu[1:]

    # --- AC flows and bus balance (Example 4)
    pf, qf, pt, qt = ac_flows(case, v, th, tau, phi)
    P, Q = bus_mismatch(case, pf, qf, pt, qt, p, q)
    wp = dt[:, None] * case.c_p * beta
    wq = dt[:, None] * case.c_q * beta
    terms["zp"] = float((wp * soft_abs(P, eps_)).sum())
    terms["zq"] = float((wq * soft_abs(Q, eps_)).sum())
    dP = wp * soft_abs_grad(P, eps_)
    dQ = wq * soft_abs_grad(Q, eps_)
    f, o = case.br_from, case.br_to
    g_pf = dP[:, f].copy()
    g_pt = dP[:, o].copy()
    g_qf = dQ[:, f].copy()
    g_qt = dQ[:, o].copy()
    gp -= sg * dP[:, case.gen_bus]
    gq -= sg * dQ[:, case.gen_bus]

    # --- thermal limit on the worse end (Example 1)
    sf = np.sqrt(pf * pf + qf * qf)
    st = np.sqrt(pt * pt + qt * qt)
    use_fr = sf >= st                      # reading: ties go to the "fr" end
    smax_end = np.where(use_fr, sf, st)
    u = smax_end - case.s_max[None, :]
    ws = dt[:, None] * case.c_s * beta
    terms["zs"] = float((ws * soft_relu(u, eps_)).sum())
    dS = ws * soft_relu_grad(u, eps_)
    with np.errstate(invalid="ignore", divide="ignore"):
        kf = np.where(use_fr & (sf > 0), dS / np.where(sf > 0, sf, 1.0), 0.0)
        kt = np.where(~use_fr & (st > 0), dS / np.where(st > 0, st, 1.0), 0.0)
    g_pf += kf * pf; g_qf += kf * qf
    g_pt += kt * pt; g_qt += kt * qt

    # --- zonal reserve shortfall
    rz = np.zeros((T, case.n_zone))
    np.add.at(rz.T, case.gen_zone, r.T)
    uz = case.reserve_req - rz
    wz = dt[:, None] * case.c_rz * beta
    terms["zrz"] = float((wz * soft_relu(uz, eps_)).sum())
    dZ = wz * soft_relu_grad(uz, eps_)
    gr -= dZ[:, case.gen_zone]

    # --- penalized linear constraints rho * sigma_s(violation): headroom and ramps; with on/off
    #     status the limits scale by u: p + r <= pmax u, p >= pmin u, qmin u <= q <= qmax u
    wr = case.rho * beta
    uon = 1.0 if uo is None else uo
    uh = p + r - case.pmax[None, :] * uon
    terms["zhead"] = float((wr * soft_relu(uh, eps_)).sum())
    dH = wr * soft_relu_grad(uh, eps_)
    gp += dH
    gr += dH
    if uo is not None:
        gu -= case.pmax * dH
        lims = ((case.pmin * uo - p, gp, -1.0, case.pmin), (q - case.qmax * uo, gq, 1.0, -case.qmax),
                (case.qmin * uo - q, gq, -1.0, case.qmin))
        for viol, gvar, sgn, cu in lims:
            terms["zhead"] += float((wr * soft_relu(viol, eps_)).sum())
            dl = wr * soft_relu_grad(viol, eps_)
            gvar += sgn * dl
            gu += cu * dl
    if T > 1:
        lim = case.ramp[None, :] * dt[1:, None]
        up = p[1:] - p[:-1] - lim
        dn = p[:-1] - p[1:] - lim
        terms["zramp"] = float((wr * (soft_relu(up, eps_) + soft_relu(dn, eps_))).sum())
        dU = wr * soft_relu_grad(up, eps_)
        dD = wr * soft_relu_grad(dn, eps_)
        gp[1:] += dU - dD
        gp[:-1] += dD - dU

    # --- contingencies (Sec. II-E)
    if net is None:
        net = dc_network(case)
    _, pbar = dc_injections(case, p)
    bflow = phase_shift_flows(case, net, branch_tau_phi(case, tau, phi)[1]) if X else None
    th_dc, fbase = dc_base_flows(case, net, pbar, bflow)
    use_qf = qf * qf >= qt * qt           # reading: the q of the worse end, ties to "fr"
    qmax2 = np.where(use_qf, qf * qf, qt * qt)
    z_ctg = np.zeros((T, case.K))
    gin_all = np.zeros((T, n))
    gq2_all = np.zeros((T, case.n_branch))
    gb_all = np.zeros((T, case.n_branch))
    if case.K > 0:
        U, den = outage_columns(case, net)                 # u_k [n-1, K], SMW denominators [K]
        plist = range(T) if periods is None else periods
        for t in plist:
            bt = None if bflow is None else bflow[t]
            if mode == "brute":
                z, gin, gq2, gb = _ctg_period_brute(case, net, pbar[t], qmax2[t], dt[t], bt)
            else:
                z, gin, gq2, gb = _ctg_period_smw(case, net, th_dc[t, net.keep], qmax2[t], dt[t], U, den, bt)
            z_ctg[t] = z
            gin_all[t] = gin
            gq2_all[t] = gq2
            gb_all[t] = gb
    terms["zctg"] = float(z_ctg.sum())
    gp += sg * gin_all[:, case.gen_bus]
    g_qf += np.where(use_qf, 2 * qf * gq2_all, 0.0)
    g_qt += np.where(~use_qf, 2 * qt * gq2_all, 0.0)

    # --- pull branch-end adjoints back to (v, theta, tau, phi) and gather per bus
    part = ac_flow_partials(case, v, th, tau, phi)
    gvf = g_pf * part["pf"][0] + g_qf * part["qf"][0] + g_pt * part["pt"][0] + g_qt * part["qt"][0]
    gvo = g_pf * part["pf"][1] + g_qf * part["qf"][1] + g_pt * part["pt"][1] + g_qt * part["qt"][1]
    gd = g_pf * part["pf"][2] + g_qf * part["qf"][2] + g_pt * part["pt"][2] + g_qt * part["qt"][2]
    np.add.at(gv.T, f, gvf.T)
    np.add.at(gv.T, o, gvo.T)
    np.add.at(gth.T, f, gd.T)
    np.subtract.at(gth.T, o, gd.T)

    gtau = gphi = None
    if X:
        gtb = g_pf * part["pf"][3] + g_qf * part["qf"][3] + g_pt * part["pt"][3] + g_qt * part["qt"][3]
        xf = case.xf_branch
        gtau = gtb[:, xf]
        # phi enters delta = theta_f - theta_o - phi (AC) and b = -y phi (contingency DC flows)
        gphi = -gd[:, xf] - net.y[xf][None, :] * gb_all[:, xf]
    obj = float(sum(terms.values()))
    grad = pack(gv, gth, gp, gq, gr, gtau, gphi, gu) if want_grad else None
    return Result(obj=obj, grad=grad, terms=terms, z_ctg=z_ctg, g_inj=gin_all)


def objective(case, x, **kw) -> float:
    return evaluate(case, x, want_grad=False, **kw).obj
