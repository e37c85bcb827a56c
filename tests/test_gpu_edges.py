"""Degenerate and limit-size inputs through the C ABI against the FP64 oracle: no contingencies
(K = 0, the base case alone), a single outage (K = 1), a single period (T = 1: no ramp terms), the
smallest grid (two buses, one branch, one generator, no outage possible without islanding), the
largest bus incidence the library accepts (a hub bus with 32 branch ends: one full warp-wide
segment in the balance and adjoint reductions) and the largest bid-block count it accepts (64
blocks per device, Example 3); each alone, with both DC solvers and both precisions, then all of
them in one ragged batch, and the graph-replayed Adam loop on the degenerate ones.

Tolerances as in the other parity tests: 1e-10 relative (FP64 path), 1e-4 (mixed path, with the
oracle evaluated at the same FP32-rounded point)."""
import dataclasses
import functools

import numpy as np
import pytest

import oracle
import synth
from gradcheck import check_at

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def qg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import qg as mod
    return mod


def two_bus(T=3):
    """Bus 0 holds the generator, bus 1 the load; one lossy line (r > 0) with line charging; three
    periods so that the ramp terms are present."""
    one = np.ones(1)
    lp = np.zeros((T, 2))
    lp[:, 1] = 0.5 * (1.0 + 0.2 * np.arange(T))
    return synth.Case(
        name="two", seed=0, n_bus=2, n_branch=1, n_gen=1, n_zone=1, ref_bus=0,
        br_from=np.array([0], np.int32), br_to=np.array([1], np.int32), br_r=np.array([0.02]),
        br_x=np.array([0.2]), br_b=np.array([0.04]), s_max=one * 0.6, s_max_ctg=one * 0.6,
        gen_bus=np.array([0], np.int32), gen_zone=np.array([0], np.int32), cost_a=one * 2.0, cost_b=one * 20.0,
        cost_r=one * 3.0, pmin=0 * one, pmax=one * 1.5, qmin=-one * 0.75, qmax=one * 0.75, ramp=one * 0.3,
        vmin=np.full(2, 0.9), vmax=np.full(2, 1.1), T=T, dt=np.ones(T), load_p=lp, load_q=0.329 * lp,
        reserve_req=0.1 * lp.sum(axis=1, keepdims=True), bus_zone=np.zeros(2, np.int32),
        ctg=np.zeros(0, np.int32))


def star(leaves, T=4):
    """A hub bus joined to `leaves` buses (radial, so no outage list), the generator on a leaf."""
    n, M = leaves + 1, leaves
    lp = np.full((T, n), 0.05) * (1.0 + 0.1 * np.arange(T))[:, None]
    one = np.ones(1)
    return synth.Case(
        name="star", seed=0, n_bus=n, n_branch=M, n_gen=1, n_zone=1, ref_bus=0,
        br_from=np.zeros(M, np.int32), br_to=np.arange(1, n, dtype=np.int32), br_r=np.full(M, 0.01),
        br_x=np.full(M, 0.1), br_b=np.full(M, 0.02), s_max=np.full(M, 0.3), s_max_ctg=np.full(M, 0.3),
        gen_bus=np.array([1], np.int32), gen_zone=np.array([0], np.int32), cost_a=one, cost_b=one * 15.0,
        cost_r=one * 2.0, pmin=0 * one, pmax=one * 4.0, qmin=-one * 2.0, qmax=one * 2.0, ramp=one * 1.2,
        vmin=np.full(n, 0.9), vmax=np.full(n, 1.1), T=T, dt=np.ones(T), load_p=lp, load_q=0.329 * lp,
        reserve_req=0.1 * lp.sum(axis=1, keepdims=True), bus_zone=np.zeros(n, np.int32),
        ctg=np.zeros(0, np.int32))


@functools.lru_cache(maxsize=None)
def case_named(name):
    c = synth.tiny()
    if name == "tiny_k0":
        return dataclasses.replace(c, name="tiny_k0", ctg=np.zeros(0, np.int32))
    if name == "tiny_t1":
        return dataclasses.replace(c, name="tiny_t1", T=1, dt=c.dt[:1], load_p=c.load_p[2:3],
                                   load_q=c.load_q[2:3], reserve_req=c.reserve_req[2:3])
    if name == "two_bus":
        return two_bus()
    if name == "star32":
        return star(32)
    if name == "mid_k1":
        m = synth.mid()
        return dataclasses.replace(m, name="mid_k1", ctg=m.ctg[:1].copy())
    if name == "tiny_b64":
        return synth.with_commitment(synth.with_block_bids(c, 64, 0.3, 5), seed=5)
    raise KeyError(name)


NAMES = ["tiny_k0", "tiny_t1", "two_bus", "star32", "mid_k1", "tiny_b64"]


def start(c, seed):
    x = synth.random_point(c, seed)
    lo, hi = oracle.box(c)
    return np.clip(x, lo, hi)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grel(g, gr):
    return np.linalg.norm(g - gr) / np.linalg.norm(gr)


def as_f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def gpu_eval(qg, cases, x, precision, **kw):
    s = qg.Solver(cases, precision=precision, **kw)
    xt = torch.tensor(x, dtype=s.dtype, device="cuda")
    obj, g = s.eval_grad(xt)
    torch.cuda.synchronize()
    out = (obj.cpu().numpy().copy(), g.double().cpu().numpy().copy(), s.breakdown())
    s.close()
    return out


def test_edge_cases_are_what_they_claim():
    assert len(case_named("tiny_k0").ctg) == 0 and len(case_named("mid_k1").ctg) == 1
    assert case_named("tiny_t1").T == 1
    c = case_named("two_bus")
    assert (c.n_bus, c.n_branch, c.n_gen) == (2, 1, 1)
    assert np.sum(case_named("star32").br_from == 0) == 32
    assert case_named("tiny_b64").blk_width.shape[1] == 64


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("dc", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_edge_case_parity(qg, name, dc, precision):
    c = case_named(name)
    x = start(c, 11)
    tol = TOL64 if precision == 0 else TOL32
    if precision == 1:
        x = as_f32(x)
    obj, g, terms = gpu_eval(qg, c, x, precision, dc_solver=dc)
    ref = oracle.evaluate(c, x)
    assert rel(obj[0], ref.obj) <= tol, (obj[0], ref.obj)
    check_at(g, ref.grad, c, tol)
    for k, term in enumerate(oracle.TERM_NAMES):
        assert abs(terms[0, k] - ref.terms[term]) <= tol * max(abs(ref.terms[term]), 1e-6 * abs(ref.obj)), term
    if len(c.ctg) == 0:
        assert terms[0, oracle.TERM_NAMES.index("zctg")] == 0.0
    if c.T == 1:
        assert terms[0, oracle.TERM_NAMES.index("zramp")] == 0.0


@pytest.mark.parametrize("precision", [0, 1])
def test_edge_cases_in_one_ragged_batch(qg, precision):
    cases = [case_named(n) for n in NAMES]
    xs = [start(c, 20 + i) for i, c in enumerate(cases)]
    tol = TOL64 if precision == 0 else TOL32
    if precision == 1:
        xs = [as_f32(x) for x in xs]
    obj, g, _ = gpu_eval(qg, cases, np.concatenate(xs), precision)
    o = 0
    for b, (c, x) in enumerate(zip(cases, xs)):
        ref = oracle.evaluate(c, x)
        assert rel(obj[b], ref.obj) <= tol, (c.name, obj[b], ref.obj)
        check_at(g[o:o + c.n_x], ref.grad, c, tol, c.name)
        o += c.n_x
    assert o == g.size


@pytest.mark.parametrize("name", ["tiny_k0", "tiny_t1", "two_bus", "star32"])
def test_edge_case_solve_trajectory(qg, name):
    """qg_solve (graph replay of evaluation + fused Adam) against the oracle's own loop."""
    c = case_named(name)
    x0 = start(c, 5)
    iters = 20
    s = qg.Solver(c, precision=qg.QG_FP64)
    xt = torch.tensor(x0, dtype=torch.float64, device="cuda")
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
    qg.qg_solve(s.h, xt, iters, 1e-3, 0.9, 0.999, trace)
    torch.cuda.synchronize()
    lo, hi = oracle.box(c)
    x, m, v = x0.copy(), np.zeros_like(x0), np.zeros_like(x0)
    tr = trace.cpu().numpy()
    for i in range(1, iters + 1):
        ref = oracle.evaluate(c, x)
        assert rel(tr[i - 1], ref.obj) <= 1e-9, (i, tr[i - 1], ref.obj)
        x, m, v = oracle.adam_step(x, m, v, ref.grad, i, 1e-3, 0.9, 0.999, 1e-8, lo, hi)
    xg = xt.cpu().numpy()
    assert np.max(np.abs(xg - x)) <= 1e-9
    assert np.all(xg >= lo) and np.all(xg <= hi)
    s.close()
