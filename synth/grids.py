"""Seeded synthetic AC unit-commitment cases.

This module only draws inputs: topology, branch and generator parameters, load
profiles, reserve requirements and contingency lists.  It holds none of the
solver's arithmetic (no power flow, no penalty, no derivative), so the FP64
oracle and the CUDA path can both consume its cases without sharing method code.

The C3E3.1 cases the paper runs on (Sec. IV) are not available, so these grids
stand in for them with the shapes of the paper's workloads: a 617-bus,
18-period real-time case with 562 single-branch contingencies (Fig. 1), batches
of smaller grids, and a 23,643-bus, 48-period day-ahead case (Sec. I).

Topology recipe: a random recursive tree (bus i attaches to a uniformly drawn
earlier bus), then ceil(L/2) chords pairing the tree's L leaves in DFS order
(leaf i with leaf i + floor(L/2)), which makes the tree 2-edge-connected, then
uniform random chords up to the requested branch count.  A bridge check
(iterative Tarjan low-link) confirms that no single outage islands the grid
(the islanding restriction noted beside the MINLP of Sec. II-B).  Bus labels are
then shuffled.

Thermal ratings of the named cases are read from synth/ratings/<name>.npy,
written offline by oracle/make_ratings.py (2 x the largest merit-order DC
flow of each branch over the horizon, at least 0.5 pu).  Cases without a stored
file (ad-hoc test grids) fall back to a KCL transport proxy: with every
generator dispatched in proportion to its Pmax, each tree edge is rated for the
net injection of the subtree below it (pure KCL, no impedances) and chords for a
fraction of the median tree rating.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import List, Optional

import numpy as np

_RATINGS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ratings")


@dataclasses.dataclass
class Case:
    """One synthetic instance.  Per-unit quantities on a 100 MVA base, 1 h periods."""

    name: str
    seed: int
    # network
    n_bus: int
    n_branch: int
    n_gen: int
    n_zone: int
    ref_bus: int
    br_from: np.ndarray  # int32 [M]
    br_to: np.ndarray  # int32 [M]
    br_r: np.ndarray  # [M] series resistance
    br_x: np.ndarray  # [M] series reactance
    br_b: np.ndarray  # [M] total line charging susceptance b_ch
    s_max: np.ndarray  # [M] base-case apparent power limit
    s_max_ctg: np.ndarray  # [M] post-contingency limit
    gen_bus: np.ndarray  # int32 [G]
    gen_zone: np.ndarray  # int32 [G]
    cost_a: np.ndarray  # [G] $/pu^2 h
    cost_b: np.ndarray  # [G] $/pu h
    cost_r: np.ndarray  # [G] reserve offer $/pu h
    pmin: np.ndarray
    pmax: np.ndarray
    qmin: np.ndarray
    qmax: np.ndarray
    ramp: np.ndarray  # [G] pu per hour
    vmin: np.ndarray  # [n]
    vmax: np.ndarray  # [n]
    # horizon
    T: int
    dt: np.ndarray  # [T] hours
    load_p: np.ndarray  # [T, n]
    load_q: np.ndarray  # [T, n]
    reserve_req: np.ndarray  # [T, Z]
    bus_zone: np.ndarray  # int32 [n]
    # contingencies
    ctg: np.ndarray  # int32 [K] outaged branch ids
    # transformers (tap ratio tau, phase shift phi per period as variables; none by default)
    xf_branch: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))  # [X] branch ids
    tau_min: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))  # [X]
    tau_max: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    phi_min: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))  # [X] rad
    phi_max: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    # devices: producers by default; consumers draw p, q (balance sign +) and earn their bid value.
    # Block bids (Example 3): blk_price[g, l] per pu over blocks of width blk_width[g, l]; devices
    # without blocks (all widths 0) use the quadratic cost a p^2 + b p.
    dev_cons: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, bool))  # [G]
    blk_price: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 0)))  # [G, L]
    blk_width: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 0)))  # [G, L]
    # on/off status (Example 2): with commit, per-period variables u in [0, 1] (relaxed binaries), an
    # on cost c_on per hour, startup / shutdown costs c_su, c_sd per event, u_init before period 0
    commit: bool = False
    c_on: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))  # [G]
    c_su: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    c_sd: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    u_init: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    # penalty prices / smoothing (chosen readings; the paper does not state them)
    c_p: float = 1e4
    c_q: float = 1e4
    c_s: float = 1e3
    c_rz: float = 1e3
    rho: float = 1e3
    eps: float = 1e-3
    beta: float = 1.0

    @property
    def K(self) -> int:
        return int(self.ctg.shape[0])

    @property
    def n_xf(self) -> int:
        return int(self.xf_branch.shape[0])

    @property
    def n_cons(self) -> int:
        return int(np.count_nonzero(self.dev_cons))

    @property
    def n_x(self) -> int:
        return self.T * (2 * self.n_bus + 3 * self.n_gen + 2 * self.n_xf + (self.n_gen if self.commit else 0))

    def offsets(self):
        """Start of the v, theta, p, q, r blocks in x (each block is T rows, period-major)."""
        n, G, T = self.n_bus, self.n_gen, self.T
        return (0, T * n, 2 * T * n, 2 * T * n + T * G, 2 * T * n + 2 * T * G)

    def offsets_xf(self):
        """Start of the tau and phi blocks (T x X each), after r."""
        o = self.T * (2 * self.n_bus + 3 * self.n_gen)
        return (o, o + self.T * self.n_xf)

    def offset_u(self):
        """Start of the on-status block u (T x G, after phi; empty without commit)."""
        return self.T * (2 * self.n_bus + 3 * self.n_gen + 2 * self.n_xf)

    def flat_start(self, p: Optional[np.ndarray] = None, r: Optional[np.ndarray] = None) -> np.ndarray:
        """x with v = 1, theta = 0, q = 0 and the given dispatch (default: Pmax-proportional)."""
        T, n, G = self.T, self.n_bus, self.n_gen
        x = np.zeros(self.n_x)
        ov, ot, op, oq, orr = self.offsets()
        x[ov:ov + T * n] = 1.0
        if p is None:
            p = proportional_dispatch(self)
        x[op:op + T * G] = np.asarray(p, dtype=np.float64).reshape(T * G)
        if r is not None:
            x[orr:orr + T * G] = np.asarray(r, dtype=np.float64).reshape(T * G)
        otau, _ = self.offsets_xf()
        x[otau:otau + T * self.n_xf] = 1.0  # tau = 1, phi = 0
        if self.commit:
            x[self.offset_u():] = 1.0  # every device on
        return x


def lp_start(case: Case):
    """(x0, bound): the stored copper-plate start of a named case (flat voltage, zero angles and q,
    copper-plate p and r) and its copper-plate bound.  Written by oracle/make_ratings.py."""
    path = os.path.join(_RATINGS_DIR, case.name + "_lp.npz")
    if not os.path.exists(path):
        raise FileNotFoundError(f"no stored copper-plate start for {case.name}")
    d = np.load(path)
    return case.flat_start(d["p"], d["r"]), float(d["bound"])


def proportional_dispatch(case: Case) -> np.ndarray:
    """Each generator covers total load in proportion to its Pmax (a data recipe, not a solve)."""
    share = case.pmax / case.pmax.sum()
    return case.load_p.sum(axis=1)[:, None] * share[None, :]


# --------------------------------------------------------------------------------------------
# topology helpers (graph only)
# --------------------------------------------------------------------------------------------

def _random_tree(n: int, rng: np.random.Generator) -> np.ndarray:
    parent = np.full(n, -1, dtype=np.int64)
    for i in range(1, n):
        parent[i] = rng.integers(0, i)
    return parent


def _dfs_leaves(n: int, parent: np.ndarray) -> List[int]:
    children: List[List[int]] = [[] for _ in range(n)]
    for i in range(1, n):
        children[parent[i]].append(i)
    deg = np.zeros(n, dtype=np.int64)
    for i in range(1, n):
        deg[i] += 1
        deg[parent[i]] += 1
    leaves: List[int] = []
    stack = [0]
    while stack:
        u = stack.pop()
        if deg[u] == 1:
            leaves.append(u)
        for c in reversed(children[u]):
            stack.append(c)
    return leaves


def find_bridges(n: int, frm: np.ndarray, to: np.ndarray) -> List[int]:
    """Branch ids whose removal disconnects the graph (iterative Tarjan low-link)."""
    adj: List[List[tuple]] = [[] for _ in range(n)]
    for j, (a, b) in enumerate(zip(frm.tolist(), to.tolist())):
        adj[a].append((b, j))
        adj[b].append((a, j))
    disc = [-1] * n
    low = [0] * n
    bridges: List[int] = []
    timer = 0
    for root in range(n):
        if disc[root] != -1:
            continue
        disc[root] = low[root] = timer
        timer += 1
        stack = [(root, -1, iter(adj[root]))]
        while stack:
            u, pe, it = stack[-1]
            advanced = False
            for (w, j) in it:
                if j == pe:
                    continue
                if disc[w] == -1:
                    disc[w] = low[w] = timer
                    timer += 1
                    stack.append((w, j, iter(adj[w])))
                    advanced = True
                    break
                low[u] = min(low[u], disc[w])
            if not advanced:
                stack.pop()
                if stack:
                    p = stack[-1][0]
                    low[p] = min(low[p], low[u])
                    if low[u] > disc[p]:
                        bridges.append(pe)
    return bridges


def _multi_source_bfs(n: int, frm: np.ndarray, to: np.ndarray, seeds: np.ndarray) -> np.ndarray:
    adj: List[List[int]] = [[] for _ in range(n)]
    for a, b in zip(frm.tolist(), to.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    zone = np.full(n, -1, dtype=np.int32)
    queue = []
    for z, s in enumerate(seeds.tolist()):
        zone[s] = z
        queue.append(s)
    head = 0
    while head < len(queue):
        u = queue[head]
        head += 1
        for w in adj[u]:
            if zone[w] < 0:
                zone[w] = zone[u]
                queue.append(w)
    return zone


# --------------------------------------------------------------------------------------------
# the generator
# --------------------------------------------------------------------------------------------

def _stored_ratings(name: str, M: int) -> Optional[np.ndarray]:
    """Ratings of a named case, sized offline from its merit-order DC flows (float32 on disk)."""
    path = os.path.join(_RATINGS_DIR, name + ".npy")
    if not os.path.exists(path):
        return None
    r = np.load(path).astype(np.float64)
    if r.shape != (M,):
        raise ValueError(f"stored ratings {path} do not match the case ({r.shape} vs {M})")
    return r

def make_case(name: str, n_bus: int, n_branch: int, n_gen: int, T: int, K: int, n_zone: int = 1,
              seed: int = 0, rating_scale: float = 1.0, chord_factor: float = 0.5,
              all_branches_ctg: bool = False) -> Case:
    rng = np.random.default_rng(seed)
    n = n_bus
    if n_branch < n - 1:
        raise ValueError("need at least a spanning tree")
    # --- topology -------------------------------------------------------------------------
    for _attempt in range(64):
        parent = _random_tree(n, rng)
        leaves = _dfs_leaves(n, parent)
        L = len(leaves)
        n_leaf_chords = (L + 1) // 2 if L > 1 else 0
        if (n - 1) + n_leaf_chords <= n_branch:
            break
    else:
        raise ValueError("could not draw a tree whose leaf pairing fits the branch budget")
    edges = [(int(parent[i]), i) for i in range(1, n)]
    tree_edge_count = len(edges)
    existing = set((min(a, b), max(a, b)) for a, b in edges)
    half = L // 2
    for i in range(n_leaf_chords):
        a, b = leaves[i], leaves[(i + half) % L]
        key = (min(a, b), max(a, b))
        if a != b and key not in existing:
            existing.add(key)
            edges.append((a, b))
    while len(edges) < n_branch:
        a, b = (int(v) for v in rng.integers(0, n, size=2))
        key = (min(a, b), max(a, b))
        if a == b or key in existing:
            continue
        existing.add(key)
        edges.append((a, b))
    frm = np.array([e[0] for e in edges], dtype=np.int64)
    to = np.array([e[1] for e in edges], dtype=np.int64)
    if find_bridges(n, frm, to):
        raise ValueError("generated grid has bridges")
    M = len(edges)
    # --- branch parameters -----------------------------------------------------------------
    br_r = rng.uniform(0.005, 0.05, M)
    br_x = br_r * rng.uniform(3.0, 10.0, M)
    br_b = rng.uniform(0.0, 0.05, M)
    # --- generators ------------------------------------------------------------------------
    gen_bus = rng.choice(n, size=n_gen, replace=False).astype(np.int64)
    cost_a = rng.uniform(0.01, 0.1, n_gen)
    cost_b = rng.uniform(10.0, 40.0, n_gen)
    pmax = rng.uniform(0.5, 3.0, n_gen)
    pmin = np.zeros(n_gen)
    ramp = 0.3 * pmax
    qmin = -0.5 * pmax
    qmax = 0.5 * pmax
    cost_r = rng.uniform(1.0, 5.0, n_gen)
    # --- loads -----------------------------------------------------------------------------
    base = rng.uniform(0.1, 0.6, n)
    prof = 1.0 + 0.15 * np.sin(2.0 * math.pi * np.arange(T) / T)
    peak = base.sum() * prof.max()
    scale = min(1.0, 0.7 * pmax.sum() / (1.1 * peak))
    load_p = (base * scale)[None, :] * prof[:, None]
    load_q = 0.329 * load_p
    # --- zones -----------------------------------------------------------------------------
    if n_zone == 1:
        bus_zone = np.zeros(n, dtype=np.int32)
    else:
        seeds = rng.choice(n, size=n_zone, replace=False)
        bus_zone = _multi_source_bfs(n, frm, to, seeds)
    gen_zone = bus_zone[gen_bus].astype(np.int32)
    reserve_req = np.zeros((T, n_zone))
    for z in range(n_zone):
        reserve_req[:, z] = 0.10 * load_p[:, bus_zone == z].sum(axis=1)
    # --- contingencies ---------------------------------------------------------------------
    if all_branches_ctg:
        ctg = np.arange(M, dtype=np.int64)
    else:
        ctg = np.sort(rng.choice(M, size=K, replace=False)).astype(np.int64)
    # --- ratings: KCL subtree transport proxy on the spanning tree -------------------------
    share = pmax / pmax.sum()
    gen_p = load_p.sum(axis=1)[:, None] * share[None, :]  # [T, G]
    inj = -load_p.copy()
    np.add.at(inj, (slice(None), gen_bus), gen_p)
    order = []  # children before parents: reverse of a BFS from the root
    children: List[List[int]] = [[] for _ in range(n)]
    for i in range(1, n):
        children[parent[i]].append(i)
    stack = [0]
    while stack:
        u = stack.pop()
        order.append(u)
        stack.extend(children[u])
    sub = inj.copy()  # [T, n] subtree sums
    for u in reversed(order):
        if u != 0:
            sub[:, parent[u]] += sub[:, u]
    s_max = np.empty(M)
    tree_rating = np.maximum(0.1, rating_scale * np.abs(sub[:, 1:]).max(axis=0))
    s_max[:tree_edge_count] = tree_rating
    s_max[tree_edge_count:] = max(0.1, rating_scale * chord_factor * float(np.median(tree_rating)))
    # --- shuffle bus labels so that index order carries no structure -----------------------
    perm = rng.permutation(n)  # old label -> new label
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    frm, to = perm[frm], perm[to]
    gen_bus = perm[gen_bus]
    load_p = load_p[:, inv]
    load_q = load_q[:, inv]
    bus_zone = bus_zone[inv]
    vmin = np.full(n, 0.9)
    vmax = np.full(n, 1.1)
    stored = _stored_ratings(name, M)
    if stored is not None:
        s_max = stored
    return Case(
        name=name, seed=seed, n_bus=n, n_branch=M, n_gen=n_gen, n_zone=n_zone, ref_bus=0,
        br_from=frm.astype(np.int32), br_to=to.astype(np.int32), br_r=br_r, br_x=br_x, br_b=br_b,
        s_max=s_max, s_max_ctg=s_max.copy(), gen_bus=gen_bus.astype(np.int32),
        gen_zone=gen_zone.astype(np.int32), cost_a=cost_a, cost_b=cost_b, cost_r=cost_r,
        pmin=pmin, pmax=pmax, qmin=qmin, qmax=qmax, ramp=ramp, vmin=vmin, vmax=vmax,
        T=T, dt=np.ones(T), load_p=load_p, load_q=load_q, reserve_req=reserve_req,
        bus_zone=bus_zone.astype(np.int32), ctg=ctg.astype(np.int32))


# --------------------------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------------------------

def tiny(seed: int = 0) -> Case:
    """14 buses, 20 branches (13 tree + 7 chords), 5 generators, 4 periods, all 20 outages."""
    return make_case("tiny14", 14, 20, 5, T=4, K=20, seed=seed, rating_scale=0.8, all_branches_ctg=True)


def rt617(seed: int = 617) -> Case:
    """617 buses, ~900 branches, 90 generators, 18 periods, 562 outages (real-time shape)."""
    return make_case("rt617", 617, 900, 90, T=18, K=562, seed=seed, rating_scale=0.8)


def mid(seed: int = 73) -> Case:
    """A mid-size case spanning several kernel tiles with ragged tails (parity workhorse)."""
    return make_case("mid150", 150, 219, 22, T=5, K=40, seed=seed, rating_scale=0.8)


BATCH_SHAPES = [(73, 12), (200, 18), (617, 24), (1576, 48)]


def batch(first_seed: int = 1000, per_shape: int = 8) -> List[Case]:
    """Uneven instances: per_shape grids of each (buses, periods) shape; M~1.46n, G~0.146n, K=ceil(0.1M)."""
    cases = []
    s = first_seed
    for (n, T) in BATCH_SHAPES:
        for _ in range(per_shape):
            M = int(round(1.46 * n))
            G = max(2, int(round(0.146 * n)))
            K = int(math.ceil(0.1 * M))
            cases.append(make_case(f"b{n}_{T}_{s}", n, M, G, T=T, K=K, seed=s, rating_scale=0.8))
            s += 1
    return cases


def dayahead(seed: int = 23643) -> Case:
    """23,643 buses, 35,000 branches, 3,000 generators, 8 zones, 48 periods, 2,000 outages."""
    return make_case("da23643", 23643, 35000, 3000, T=48, K=2000, n_zone=8, seed=seed, rating_scale=0.8)


def with_loads(case: Case, load_p: np.ndarray) -> Case:
    """The same network under another active-load profile (T x n): reactive load and zonal reserve
    requirements follow the recipe of make_case (q = 0.329 p, 10% of each zone's load)."""
    load_p = np.asarray(load_p, dtype=np.float64).reshape(case.T, case.n_bus)
    reserve = np.zeros((case.T, case.n_zone))
    for z in range(case.n_zone):
        reserve[:, z] = 0.10 * load_p[:, case.bus_zone == z].sum(axis=1)
    return dataclasses.replace(case, load_p=load_p, load_q=0.329 * load_p, reserve_req=reserve)


def with_transformers(case: Case, frac: float = 0.15, seed: int = 0) -> Case:
    """The same case with a random fraction of its branches turned into transformers: tap ratio
    tau in [0.9, 1.1]; half of them also phase shifters with phi in [-0.3, 0.3] rad (phi fixed at 0
    for the others).  tau = 1 and phi = 0 reproduce the original network."""
    rng = np.random.default_rng(seed)
    X = max(1, int(round(frac * case.n_branch)))
    xf = np.sort(rng.choice(case.n_branch, size=X, replace=False)).astype(np.int32)
    shifter = rng.random(X) < 0.5
    return dataclasses.replace(case, name=case.name + "_xf", xf_branch=xf, tau_min=np.full(X, 0.9),
                               tau_max=np.full(X, 1.1), phi_min=np.where(shifter, -0.3, 0.0),
                               phi_max=np.where(shifter, 0.3, 0.0))


def with_block_bids(case: Case, n_blocks: int = 3, cons_frac: float = 0.3, seed: int = 0) -> Case:
    """The same case with block bids (Example 3) on every device and a fraction of the buses given a
    dispatchable consumer: each producer's [0, Pmax] split into n_blocks blocks of rising price (a
    convex cost); consumers take part of their bus's load, p in [0, 1.2 x that part] bid in blocks of
    falling value (a concave value), with q = 0.329 p bounds; the fixed load of those buses drops by
    the consumers' nominal share."""
    rng = np.random.default_rng(seed)
    G, n, T = case.n_gen, case.n_bus, case.T
    nc = max(1, int(round(cons_frac * n)))
    cbus = np.sort(rng.choice(n, size=nc, replace=False)).astype(np.int32)
    share = rng.uniform(0.2, 0.5, size=nc)
    nominal = case.load_p[:, cbus].max(axis=0) * share
    load_p = case.load_p.copy()
    load_p[:, cbus] *= (1.0 - share)[None, :]
    load_q = 0.329 * load_p
    L = n_blocks
    width = np.zeros((G + nc, L))
    price = np.zeros((G + nc, L))
    width[:G] = case.pmax[:, None] / L
    base = case.cost_b + case.cost_a * case.pmax / L
    steps = np.cumsum(rng.uniform(1.0, 8.0, size=(G, L)), axis=1)
    price[:G] = base[:, None] + steps
    cmax = 1.2 * nominal
    width[G:] = cmax[:, None] / L
    price[G:] = rng.uniform(60.0, 90.0, size=nc)[:, None] - np.cumsum(rng.uniform(2.0, 10.0, size=(nc, L)), axis=1)
    cat = lambda a, b: np.concatenate([a, b])
    return dataclasses.replace(
        case, name=case.name + "_bids", n_gen=G + nc, gen_bus=cat(case.gen_bus, cbus),
        gen_zone=cat(case.gen_zone, case.bus_zone[cbus]).astype(np.int32), cost_a=cat(case.cost_a, np.zeros(nc)),
        cost_b=cat(case.cost_b, np.zeros(nc)), cost_r=cat(case.cost_r, np.zeros(nc)), pmin=cat(case.pmin, np.zeros(nc)),
        pmax=cat(case.pmax, cmax), qmin=cat(case.qmin, np.zeros(nc)), qmax=cat(case.qmax, 0.329 * cmax),
        ramp=cat(case.ramp, cmax), load_p=load_p, load_q=load_q,
        dev_cons=cat(np.zeros(G, bool), np.ones(nc, bool)), blk_price=price, blk_width=width)


def with_commitment(case: Case, seed: int = 0, off_frac: float = 0.2) -> Case:
    """The same case with on/off status variables (Example 2): per device an on cost of 1-5 $/h per
    pu of Pmax, startup cost of 10-40 and shutdown cost of 0-10 $ per pu of Pmax, and a fraction
    off_frac of the devices off before period 0."""
    rng = np.random.default_rng(seed)
    G = case.n_gen
    scale = np.maximum(case.pmax, 1e-3)
    u_init = (rng.uniform(size=G) >= off_frac).astype(np.float64)
    return dataclasses.replace(
        case, name=case.name + "_uc", commit=True, c_on=rng.uniform(1.0, 5.0, G) * scale,
        c_su=rng.uniform(10.0, 40.0, G) * scale, c_sd=rng.uniform(0.0, 10.0, G) * scale, u_init=u_init)


def horizon_slice(case: Case, t0: int, t1: int) -> Case:
    """The same network over periods [t0, t1) of the horizon only."""
    return dataclasses.replace(case, T=t1 - t0, dt=case.dt[t0:t1].copy(), load_p=case.load_p[t0:t1].copy(),
                               load_q=case.load_q[t0:t1].copy(), reserve_req=case.reserve_req[t0:t1].copy())


def load_profiles(case: Case, count: int, seed: int) -> np.ndarray:
    """Warm-start training profiles: load * U(0.8, 1.2) per profile * (1 + N(0, 0.05)) per bus, >= 0."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, case.T, case.n_bus))
    for c in range(count):
        s = rng.uniform(0.8, 1.2)
        noise = 1.0 + rng.normal(0.0, 0.05, case.n_bus)
        out[c] = np.maximum(case.load_p * s * noise[None, :], 0.0)
    return out


def random_point(case: Case, seed: int, spread: float = 1.0) -> np.ndarray:
    """A random x inside the box: v in [vmin, vmax], theta ~ N(0, 0.1 spread), p, q, r, tau, phi uniform."""
    rng = np.random.default_rng(seed)
    T, n, G = case.T, case.n_bus, case.n_gen
    v = rng.uniform(case.vmin, case.vmax, size=(T, n))
    th = rng.normal(0.0, 0.1 * spread, size=(T, n))
    th[:, case.ref_bus] = 0.0
    p = rng.uniform(case.pmin, case.pmax, size=(T, G))
    q = rng.uniform(case.qmin, case.qmax, size=(T, G))
    r = rng.uniform(0.0, 0.3, size=(T, G)) * case.pmax
    if case.n_cons:
        r[:, case.dev_cons] = 0.0  # consumers hold no reserve
    parts = [v.ravel(), th.ravel(), p.ravel(), q.ravel(), r.ravel()]
    if case.n_xf:
        parts.append(rng.uniform(case.tau_min, case.tau_max, size=(T, case.n_xf)).ravel())
        parts.append(rng.uniform(case.phi_min, case.phi_max, size=(T, case.n_xf)).ravel())
    if case.commit:
        parts.append(rng.uniform(0.0, 1.0, size=(T, G)).ravel())
    return np.concatenate(parts)
