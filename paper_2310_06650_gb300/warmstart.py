"""Learned warm start for the Adam solve (the AI-systems addition): generate solves with the
library itself, train the MLP on them with the library's own kernels, and compare the time to a
target objective from the learned start (mixed precision) against plain FP64 Adam from the
copper-plate start.

Host-side pieces here are orchestration and the copper-plate start of Sec. III-A (merit-order
dispatch per period, which is that projection without ramps and reserves); every evaluation,
Adam step, MLP forward and backward runs in libqg's CUDA kernels.
"""
from __future__ import annotations

import dataclasses
import time
from typing import List, Sequence

import numpy as np

from . import qg

BATCH = 32  # instances per handle


# ------------------------------------------------------------------------------------------------
# copper-plate start (Sec. III-A without ramp and reserve terms)
# ------------------------------------------------------------------------------------------------

def merit_order_dispatch(case) -> np.ndarray:
    """Per period, the least-cost dispatch meeting total load: p_g = clip((lam - b_g)/(2 a_g), pmin, pmax)
    with lam found by bisection (KKT of the separable quadratic cost)."""
    a, b = case.cost_a, case.cost_b
    out = np.zeros((case.T, case.n_gen))
    for t in range(case.T):
        L = case.load_p[t].sum()
        lo, hi = 0.0, float(b.max() + 2 * (a * case.pmax).max()) + 1.0
        for _ in range(100):
            lam = 0.5 * (lo + hi)
            if np.clip((lam - b) / (2 * a), case.pmin, case.pmax).sum() < L:
                lo = lam
            else:
                hi = lam
        out[t] = np.clip((0.5 * (lo + hi) - b) / (2 * a), case.pmin, case.pmax)
    return out


def merit_order_bound(case) -> float:
    """sum_t d_t sum_g (a p^2 + b p) at the merit-order dispatch: a lower bound of the objective
    scored with eps = 0 (dropping the reserve, ramp and network terms only removes non-negative
    penalties, and unserved load costs at least c^p per pu, far above any marginal cost)."""
    p = merit_order_dispatch(case)
    return float((case.dt[:, None] * (case.cost_a * p * p + case.cost_b * p)).sum())


def start_point(case) -> np.ndarray:
    """x0: flat voltage, zero angles and q, merit-order p, reserve spread over headroom per zone."""
    p = merit_order_dispatch(case)
    r = np.zeros_like(p)
    head = np.maximum(case.pmax[None, :] - p, 0.0)
    for z in range(case.n_zone):
        gz = case.gen_zone == z
        tot = head[:, gz].sum(axis=1, keepdims=True)
        frac = np.where(tot > 0, case.reserve_req[:, z:z + 1] / np.maximum(tot, 1e-30), 0.0)
        r[:, gz] = head[:, gz] * np.minimum(frac, 1.0)
    return case.flat_start(p, r)


# ------------------------------------------------------------------------------------------------
# features and targets
# ------------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Scaling:
    """The network learns a correction to the copper-plate start: target = (x* - x0) / scale,
    inputs are relative load deviations from the nominal profile."""
    x_scale: np.ndarray
    load_ref: np.ndarray  # T x n nominal load

    @staticmethod
    def for_case(case) -> "Scaling":
        T, n, G = case.T, case.n_bus, case.n_gen
        pm = np.tile(case.pmax, T)
        scale = np.concatenate([np.full(T * n, 0.05), np.full(T * n, 0.2), pm, pm, pm])
        return Scaling(scale, case.load_p.copy())

    def features(self, load_p: np.ndarray) -> np.ndarray:
        return (4.0 * (np.asarray(load_p) / np.maximum(self.load_ref, 1e-9) - 1.0)).reshape(len(load_p), -1)

    def to_target(self, x: np.ndarray, x0: np.ndarray) -> np.ndarray:
        return (x - x0) / self.x_scale

    def to_x(self, y: np.ndarray, x0: np.ndarray) -> np.ndarray:
        return x0 + y * self.x_scale


def clip_box(case, x: np.ndarray) -> np.ndarray:
    T, n, G = case.T, case.n_bus, case.n_gen
    v, th, p, q, r = np.split(x, [T * n, 2 * T * n, 2 * T * n + T * G, 2 * T * n + 2 * T * G])
    v = np.clip(v.reshape(T, n), case.vmin, case.vmax).ravel()
    th = th.reshape(T, n).copy()
    th[:, case.ref_bus] = 0.0
    p = np.clip(p.reshape(T, G), case.pmin, case.pmax).ravel()
    q = np.clip(q.reshape(T, G), case.qmin, case.qmax).ravel()
    r = np.clip(r.reshape(T, G), 0.0, case.pmax).ravel()
    return np.concatenate([v, th.ravel(), p, q, r])


# ------------------------------------------------------------------------------------------------
# data generation: batched Adam solves
# ------------------------------------------------------------------------------------------------

# Sec. II-F schedule used by the solves below (lr0, lrf, eps0, epsf, beta0, beta1, lag): the step size
# decays over three decades, the smoothing over four, and the homotopy scale rises from 0.1 to 1.
SCHEDULE = (1e-2, 1e-5, 5e-2, 1e-5, 0.1, 1.0, 0.25)


def schedule_table(iters: int, spec=SCHEDULE):
    """Device table (iters x 3: lr, eps, beta) of the Sec. II-F schedule, written by the library."""
    import torch
    return torch.tensor(qg.qg_schedule(iters, *spec), dtype=torch.float64, device="cuda")


def solve_many(cases: Sequence, x0s: Sequence[np.ndarray], iters: int, lr: float = 1e-3,
               precision: int = qg.QG_MIXED, schedule=None) -> List[np.ndarray]:
    """Adam solves of many instances, BATCH per handle, from the given starts; with a schedule spec,
    the Sec. II-F step-size and homotopy schedules over the iterations instead of a constant lr."""
    import torch
    out = []
    table = schedule_table(iters, schedule) if schedule else None
    for b0 in range(0, len(cases), BATCH):
        cs = list(cases[b0:b0 + BATCH])
        s = qg.Solver(cs, precision=precision)
        x = torch.tensor(np.concatenate(x0s[b0:b0 + BATCH]), dtype=s.dtype, device="cuda")
        if table is not None:
            qg.qg_solve_schedule(s.h, x, iters, table, True, 0.9, 0.999)
        else:
            qg.qg_solve(s.h, x, iters, lr, 0.9, 0.999)
        xs = x.double().cpu().numpy()
        o = 0
        for c in cs:
            out.append(xs[o:o + c.n_x].copy())
            o += c.n_x
        s.close()
    return out


# ------------------------------------------------------------------------------------------------
# training and inference
# ------------------------------------------------------------------------------------------------

class WarmStart:
    def __init__(self, case, hidden: int = 1024, max_batch: int = 64, seed: int = 0):
        import torch
        self.torch = torch
        self.case = case
        self.scaling = Scaling.for_case(case)
        self.n_in = case.T * case.n_bus
        self.n_out = case.n_x
        self.max_batch = max_batch
        self.m = qg.qg_mlp_create(self.n_in, hidden, self.n_out, max_batch, seed)
        qg.qg_mlp_set_stream(self.m, torch.cuda.current_stream().cuda_stream)
        # start from a near-zero correction: shrink the output layer's initial weights
        w = torch.zeros(qg.qg_mlp_num_params(self.m), dtype=torch.float32, device="cuda")
        qg.qg_mlp_get_params(self.m, w)
        o3 = hidden * self.n_in + hidden + hidden * hidden + hidden
        w[o3:o3 + self.n_out * hidden] *= 0.01
        qg.qg_mlp_set_params(self.m, w)

    def train(self, load_profiles: np.ndarray, starts: Sequence[np.ndarray], solutions: Sequence[np.ndarray],
              epochs: int, batch: int = 64, lr: float = 1e-3, seed: int = 0) -> List[float]:
        torch = self.torch
        X = torch.tensor(self.scaling.features(load_profiles), dtype=torch.float32, device="cuda")
        Y = torch.tensor(np.stack([self.scaling.to_target(x, x0) for x, x0 in zip(solutions, starts)]),
                         dtype=torch.float32, device="cuda")
        n = X.shape[0]
        rng = np.random.default_rng(seed)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        hist = []
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(n), device="cuda")
            tot = 0.0
            for b0 in range(0, n - batch + 1, batch):
                idx = perm[b0:b0 + batch]
                xb = X.index_select(0, idx).contiguous()
                yb = Y.index_select(0, idx).contiguous()
                qg.qg_mlp_train_step(self.m, xb, yb, batch, lr, 0.9, 0.999, loss)
                tot += loss.item()
            hist.append(tot / max(1, n // batch))
        return hist

    def predict(self, load_profiles: np.ndarray, starts: Sequence[np.ndarray]) -> List[np.ndarray]:
        torch = self.torch
        X = torch.tensor(self.scaling.features(load_profiles), dtype=torch.float32, device="cuda")
        out = []
        for b0 in range(0, X.shape[0], self.max_batch):
            xb = X[b0:b0 + self.max_batch].contiguous()
            y = torch.zeros(xb.shape[0], self.n_out, dtype=torch.float32, device="cuda")
            qg.qg_mlp_forward(self.m, xb, xb.shape[0], y)
            for k, row in enumerate(y.double().cpu().numpy()):
                out.append(clip_box(self.case, self.scaling.to_x(row, starts[b0 + k])))
        return out

    def close(self):
        if self.m:
            qg.qg_mlp_destroy(self.m)
            self.m = None


# ------------------------------------------------------------------------------------------------
# time to a target objective
# ------------------------------------------------------------------------------------------------

def objective_eps0(scorer, x_dev) -> float:
    """Phi at eps = 0 (hard abs / ReLU), the score the target refers to."""
    obj, _ = scorer.eval_grad(x_dev)
    return float(obj[0].item())


def solve_trace(case, x0: np.ndarray, precision: int, iters: int, every: int, lr: float = 1e-3, table=None,
                t_start_ms: float = 0.0):
    """Single-instance Adam solve; returns (cumulative GPU ms after each chunk, eps = 0 objective
    after each chunk).  With a schedule table (device, rows x 3) the run follows it from its first
    row.  The scoring evaluations run on a separate FP64 handle and are not timed; t_start_ms (e.g.
    the MLP inference that produced x0) is added to every time."""
    torch = __import__("torch")
    s = qg.Solver(case, precision=precision)
    scorer = qg.Solver(case, precision=qg.QG_FP64, eps=0.0)
    x = torch.tensor(x0, dtype=s.dtype, device="cuda")
    xs = torch.zeros(case.n_x, dtype=torch.float64, device="cuda")

    def run(n, first):
        if table is not None:
            qg.qg_solve_schedule(s.h, x, n, table, first, 0.9, 0.999)
        else:
            qg.qg_solve(s.h, x, n, lr, 0.9, 0.999)

    run(every, True)  # capture the graph outside the timed chunks
    qg.qg_set_step(s.h, 0)
    x.copy_(torch.tensor(x0, dtype=s.dtype, device="cuda"))
    times, objs = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    xs.copy_(x)
    objs.append(objective_eps0(scorer, xs))
    times.append(t_start_ms)
    for k in range(0, iters, every):
        e0.record()
        run(every, k == 0)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        xs.copy_(x)
        objs.append(objective_eps0(scorer, xs))
    s.close()
    scorer.close()
    return np.cumsum(times), np.array(objs)


def time_to(times_ms: np.ndarray, objs: np.ndarray, target: float) -> float:
    hit = np.nonzero(objs <= target)[0]
    return float(times_ms[hit[0]]) if len(hit) else float("inf")


# ------------------------------------------------------------------------------------------------
# experiment driver
# ------------------------------------------------------------------------------------------------

ARMS = (("plain_fp64", "FP64 from the copper-plate start"), ("mixed_lp", "mixed from the copper-plate start"),
        ("fp64_learned", "FP64 from the learned start"), ("warm_mixed", "mixed from the learned start"))


def experiment(case, n_train: int, n_test: int, solve_iters: int, epochs: int, eval_iters: int, every: int,
               seed: int = 5000, hidden: int = 1024, schedule=SCHEDULE, warm_skip: float = 0.25,
               const_arm: bool = False, bounds=None, eval_schedule="same", target_ratio=None, log=print) -> dict:
    """Train on n_train generated solves, then for n_test held-out profiles compare four Adam arms,
    {FP64, mixed precision} x {copper-plate start, learned start}, on GPU time to a target objective
    (eps = 0 scoring).  The target is 1% above the copper-plate bound when plain FP64 Adam from the
    copper-plate start gets there within eval_iters, else 1% above the best objective that arm
    reaches.  Every arm follows the Sec. II-F schedule of eval_iters iterations (schedule=None: a
    constant lr of 1e-3); the learned-start arms enter it after the first warm_skip fraction (the
    learned start takes the place of the early large steps) and their time includes the MLP
    inference.  Held-out profiles come from their own generator (seed + 1), so they do not depend on
    n_train.  bounds: optional per-profile lower bounds of Phi (dicts with "copper_plate" and
    "contingency_bound"), against which the target is also stated; with target_ratio the target is
    target_ratio x the profile's contingency-aware bound instead.  eval_schedule: the schedule spec of
    the compared runs ("same": the training solves' schedule).  const_arm adds, for context, plain FP64
    Adam with a constant lr of 1e-3."""
    import synth
    torch = __import__("torch")
    t0 = time.time()
    prof = synth.load_profiles(case, n_train, seed)
    prof_test = synth.load_profiles(case, n_test, seed + 1)
    cases = [synth.with_loads(case, lp) for lp in prof]
    tests = [synth.with_loads(case, lp) for lp in prof_test]
    starts = [start_point(c) for c in cases]
    sols = solve_many(cases, starts, solve_iters, schedule=schedule)
    t_gen = time.time() - t0
    log(f"generated {n_train} solves in {t_gen:.1f} s")
    ws = WarmStart(case, hidden=hidden, seed=seed)
    t1 = time.time()
    hist = ws.train(prof, starts, sols, epochs)
    t_train = time.time() - t1
    log(f"trained {epochs} epochs in {t_train:.1f} s, loss {hist[0]:.4g} -> {hist[-1]:.4g}")
    espec = schedule if isinstance(eval_schedule, str) and eval_schedule == "same" else eval_schedule
    table = schedule_table(eval_iters, espec) if espec else None
    skip = int(round(warm_skip * eval_iters)) if schedule else 0
    table_b = table[skip:].contiguous() if table is not None else None
    rows = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i, c in enumerate(tests):
        bound = merit_order_bound(c)
        x_lp = start_point(c)
        e0.record()
        pred = ws.predict(prof_test[i:i + 1], [x_lp])[0]
        e1.record()
        e1.synchronize()
        t_mlp = e0.elapsed_time(e1)
        traces = {
            "plain_fp64": solve_trace(c, x_lp, qg.QG_FP64, eval_iters, every, table=table),
            "mixed_lp": solve_trace(c, x_lp, qg.QG_MIXED, eval_iters, every, table=table),
            "fp64_learned": solve_trace(c, pred, qg.QG_FP64, eval_iters - skip, every, table=table_b, t_start_ms=t_mlp),
            "warm_mixed": solve_trace(c, pred, qg.QG_MIXED, eval_iters - skip, every, table=table_b, t_start_ms=t_mlp),
        }
        ta, oa = traces["plain_fp64"]
        if target_ratio is not None and bounds is not None:
            target = target_ratio * bounds[i]["contingency_bound"]
            kind = f"{target_ratio} x the contingency-aware bound"
        else:
            target = 1.01 * bound
            kind = "1% of copper-plate bound"
            if not np.isfinite(time_to(ta, oa, target)):
                target = 1.01 * float(oa.min())
                kind = "1% above the best objective of plain FP64 Adam"
        row = {"bound": bound, "target": target, "target_kind": kind, "mlp_ms": t_mlp}
        if bounds is not None and i < len(bounds):
            row["target_over_copper_plate"] = target / bounds[i]["copper_plate"]
            row["target_over_contingency_bound"] = target / bounds[i]["contingency_bound"]
        for name, (tt, oo) in traces.items():
            row[name] = {"ms": time_to(tt, oo, target), "phi0": float(oo[0]), "best": float(oo.min()),
                         "ms_total": float(tt[-1])}
        if const_arm:
            tc, oc = solve_trace(c, x_lp, qg.QG_FP64, eval_iters, every)
            row["plain_fp64_const_lr"] = {"ms": time_to(tc, oc, target), "best": float(oc.min())}
        rows.append(row)
        log(row)
    ws.close()

    def median(arm):
        v = [r[arm]["ms"] for r in rows if np.isfinite(r[arm]["ms"])]
        return float(np.median(v)) if len(v) == len(rows) and v else None

    return {"n_train": n_train, "n_test": n_test, "solve_iters": solve_iters, "epochs": epochs,
            "eval_iters": eval_iters, "every": every, "schedule": list(schedule) if schedule else None,
            "eval_schedule": list(espec) if espec else None,
            "warm_skip": warm_skip if schedule else 0.0, "gen_s": t_gen, "train_s": t_train,
            "loss_first": hist[0], "loss_last": hist[-1], "rows": rows,
            "median_ms": {arm: median(arm) for arm, _ in ARMS},
            "reached": {arm: int(sum(np.isfinite(r[arm]["ms"]) for r in rows)) for arm, _ in ARMS},
            "warm_faster": int(sum(r["warm_mixed"]["ms"] < r["plain_fp64"]["ms"] for r in rows)),
            "reached_1pct": int(sum(r["target_kind"].startswith("1% of") for r in rows))}


def mlp_bench(case, hidden: int = 1024, batch: int = 64, reps: int = 20, seed: int = 0) -> dict:
    """Device time of the warm-start network at the case's size (input T n, output n_x): the mean of
    `reps` forward passes (x -> y: three tensor-core GEMMs and their epilogues), each after a 512 MB
    write that evicts the weights from L2, and of `reps` training steps (forward, backward, Adam,
    BF16 weight refresh).  The forward pass reads every BF16 weight once: its floor is those bytes
    at the HBM bandwidth."""
    torch = __import__("torch")
    n_in, n_out = case.T * case.n_bus, case.n_x
    m = qg.qg_mlp_create(n_in, hidden, n_out, batch, seed)
    stream = torch.cuda.current_stream()
    qg.qg_mlp_set_stream(m, stream.cuda_stream)
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(batch, n_in, generator=g).cuda()
    tgt = 0.1 * torch.randn(batch, n_out, generator=g).cuda()
    y = torch.zeros(batch, n_out, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        qg.qg_mlp_forward(m, x, batch, y)
        qg.qg_mlp_train_step(m, x, tgt, batch, 1e-4, 0.9, 0.999, loss)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for k, (a, b) in enumerate(ev):
        flush.fill_(k & 0xFF)
        a.record(stream)
        qg.qg_mlp_forward(m, x, batch, y)
        b.record(stream)
    et = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in et:
        a.record(stream)
        qg.qg_mlp_train_step(m, x, tgt, batch, 1e-4, 0.9, 0.999, loss)
        b.record(stream)
    torch.cuda.synchronize()
    qg.qg_mlp_check(m)
    qg.qg_mlp_destroy(m)
    fwd = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    train = float(np.mean([a.elapsed_time(b) for a, b in et]))
    wbytes = 2.0 * hidden * (n_in + hidden + n_out)
    return {"shape": f"{n_in} -> {hidden} -> {hidden} -> {n_out}, batch {batch}", "forward_ms": fwd,
            "train_step_ms": train, "weight_bytes_bf16": wbytes, "finite": bool(torch.isfinite(y).all().item())}


# Schedule variants for the attainable-objective study: (name, spec) with spec the qg_schedule
# arguments (lr0, lrf, eps0, epsf, beta0, beta1, lag), or None for a constant lr of 1e-3.
VARIANTS = (("default", SCHEDULE),
            ("lr0 1e-1", (1e-1, 1e-5, 5e-2, 1e-5, 0.1, 1.0, 0.25)),
            ("lr0 3e-3", (3e-3, 1e-6, 5e-2, 1e-5, 0.1, 1.0, 0.25)),
            ("no homotopy", (1e-2, 1e-5, 5e-2, 1e-5, 1.0, 1.0, 0.25)),
            ("constant lr 1e-3", None))


def attainable(case, profiles: Sequence[int], iters: int, seed: int = 5001, variants=VARIANTS,
               precision: int = qg.QG_FP64, log=print) -> dict:
    """The objective (eps = 0) that long Adam runs reach from the copper-plate start of the held-out
    profiles (synth.load_profiles(case, max(profiles) + 1, seed), the generator experiment() draws
    its held-out profiles from), under each schedule variant of `iters` iterations: per profile and
    variant the best Phi seen (scored every iters / 50 iterations) and the GPU time of the run."""
    import synth
    prof = synth.load_profiles(case, max(profiles) + 1, seed)
    every = max(1, iters // 50)
    out = []
    for i in profiles:
        c = synth.with_loads(case, prof[i])
        x0 = start_point(c)
        row = {"profile": i, "copper_plate_merit_order": merit_order_bound(c), "variants": {}}
        for name, spec in variants:
            table = schedule_table(iters, spec) if spec is not None else None
            tt, oo = solve_trace(c, x0, precision, iters, every, table=table)
            row["variants"][name] = {"best": float(oo.min()), "final": float(oo[-1]), "ms": float(tt[-1])}
            log(i, name, row["variants"][name])
        out.append(row)
    return {"iters": iters, "precision": "fp64" if precision == qg.QG_FP64 else "mixed", "rows": out,
            "variants": {name: (list(spec) if spec else "constant lr 1e-3") for name, spec in variants}}


def main(argv=None):
    import argparse
    import json
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    ap = argparse.ArgumentParser(description="learned warm start vs plain FP64 Adam")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=8)
    ap.add_argument("--solve-iters", type=int, default=5000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--eval-iters", type=int, default=20000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--hidden", type=int, default=1024)
    ap.add_argument("--warm-skip", type=float, default=0.25)
    ap.add_argument("--constant-lr", action="store_true", help="constant lr 1e-3 instead of the Sec. II-F schedule")
    ap.add_argument("--const-arm", action="store_true", help="add plain FP64 Adam at a constant lr for context")
    ap.add_argument("--attainable", type=int, default=0, metavar="ITERS",
                    help="instead: the best objective of long FP64 runs (ITERS iterations) per schedule variant")
    ap.add_argument("--profiles", type=int, default=4, help="held-out profiles for --attainable")
    ap.add_argument("--mlp-bench", action="store_true", help="instead: time the network at the rt617 size")
    ap.add_argument("--eval-variant", default=None, help="schedule variant (VARIANTS name) of the compared runs")
    ap.add_argument("--target-ratio", type=float, default=None,
                    help="target = this x the contingency-aware bound (tests/golden/rt617_ttt_bounds.json)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from .build import build
    build()
    if a.mlp_bench:
        print(json.dumps(mlp_bench(synth.rt617())))
        return
    if a.attainable:
        res = attainable(synth.rt617(), list(range(a.profiles)), a.attainable, log=lambda *s: print(*s, flush=True))
        line = json.dumps(res)
        print(line)
        if a.out:
            with open(a.out, "w") as f:
                f.write(line + "\n")
        return
    bounds = None
    bpath = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                         "rt617_ttt_bounds.json")
    if os.path.exists(bpath):
        with open(bpath) as f:
            bounds = json.load(f)["rows"]
    espec = dict(VARIANTS)[a.eval_variant] if a.eval_variant else "same"
    res = experiment(synth.rt617(), a.train, a.test, a.solve_iters, a.epochs, a.eval_iters, a.every, hidden=a.hidden,
                     schedule=None if a.constant_lr else SCHEDULE, warm_skip=a.warm_skip, const_arm=a.const_arm,
                     bounds=bounds, eval_schedule=espec, target_ratio=a.target_ratio,
                     log=lambda *s: print(*s, flush=True))
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
