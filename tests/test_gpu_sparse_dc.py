"""The sparse DC solver (QG_DC_SPARSE: LDL^T with a dense tail, gather lists, no PTDF) through the
C ABI, against the FP64 oracle and against the dense solver.  Grids: tiny14 and mid150 (every node
eliminated, no tail), rt617 (71-node tail), the 1,576-bus batch grid (189-node tail, 48 periods),
a 70-period grid (two passes over the periods), and the day-ahead grid (23,643 buses, 35,000
branches, 2,000 outages, a 3,109-node tail) where QG_DC_AUTO picks the sparse solver by itself.

Tolerances as in the other parity tests: 1e-10 relative (FP64 path), 1e-4 (mixed path, with the
oracle evaluated at the same FP32-rounded point)."""
import functools

import numpy as np
import pytest

import oracle
import synth
from gradcheck import check_at, check_grad
from oracle.copperplate import lambda_dispatch

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


@functools.lru_cache(maxsize=None)
def case_named(name):
    return {"tiny": synth.tiny, "mid": synth.mid, "rt617": synth.rt617,
            "b1576": lambda: synth.batch(per_shape=1)[-1],
            "t70": lambda: synth.make_case("t70", 400, 600, 60, T=70, K=60, seed=11, rating_scale=0.8),
            "da": synth.dayahead}[name]()


@functools.lru_cache(maxsize=None)
def dayahead_net():
    return oracle.dc_network(case_named("da"))


def start(case, seed=99, spread=0.02):
    """Merit-order dispatch with flat voltage, perturbed inside the box."""
    x = case.flat_start(lambda_dispatch(case)) + spread * (synth.random_point(case, seed) - 0.5)
    lo, hi = oracle.box(case)
    return np.clip(x, lo, hi)


def as_f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grel(g, gr):
    return np.linalg.norm(g - gr) / np.linalg.norm(gr)


def gpu_eval(qg, case, x, precision, **kw):
    s = qg.Solver(case, precision=precision, **kw)
    xt = torch.tensor(x, dtype=s.dtype, device="cuda")
    obj, g = s.eval_grad(xt)
    torch.cuda.synchronize()
    out = (obj.cpu().numpy().copy(), g.double().cpu().numpy().copy(), s.breakdown())
    s.close()
    return out


def check(res, ref, tol, case, skip_terms=()):
    obj, g, terms = res
    assert rel(obj[0], ref.obj) <= tol, (obj[0], ref.obj)
    check_at(g, ref.grad, case, tol)
    for k, name in enumerate(oracle.TERM_NAMES):
        if name in skip_terms:
            continue
        assert abs(terms[0, k] - ref.terms[name]) <= tol * max(abs(ref.terms[name]), 1e-6 * abs(ref.obj)), name


@pytest.mark.parametrize("name", ["tiny", "mid", "rt617", "b1576", "t70"])
def test_sparse_fp64_parity(qg, name):
    c = case_named(name)
    x = start(c)
    check(gpu_eval(qg, c, x, qg.QG_FP64, dc_solver=qg.QG_DC_SPARSE), oracle.evaluate(c, x), TOL64, c)


@pytest.mark.parametrize("name", ["mid", "rt617", "b1576", "t70"])
def test_sparse_mixed_parity(qg, name):
    c = case_named(name)
    x = as_f32(start(c))
    check(gpu_eval(qg, c, x, qg.QG_MIXED, dc_solver=qg.QG_DC_SPARSE), oracle.evaluate(c, x), TOL32, c)


def test_sparse_and_dense_solvers_agree(qg):
    """Same quantities, two routes (PTDF products vs factor solves): equal to rounding."""
    c = case_named("rt617")
    x = start(c, seed=5)
    od, gd, td = gpu_eval(qg, c, x, qg.QG_FP64, dc_solver=qg.QG_DC_DENSE)
    osp, gsp, tsp = gpu_eval(qg, c, x, qg.QG_FP64, dc_solver=qg.QG_DC_SPARSE)
    assert rel(osp[0], od[0]) <= 1e-12
    check_grad(gsp, gd, c, 1e-11, 1e-11)
    assert np.allclose(tsp, td, rtol=1e-11, atol=1e-9)


def test_sparse_solve_trajectory_matches_dense(qg):
    """qg_solve (graph-replayed evaluation + fused Adam) on both solvers: same iterates."""
    c = case_named("rt617")
    x0 = start(c, seed=6)
    out = {}
    for dc in (qg.QG_DC_DENSE, qg.QG_DC_SPARSE):
        s = qg.Solver(c, precision=qg.QG_FP64, dc_solver=dc)
        xt = torch.tensor(x0, dtype=torch.float64, device="cuda")
        trace = torch.zeros(25, dtype=torch.float64, device="cuda")
        qg.qg_solve(s.h, xt, 25, 1e-3, 0.9, 0.999, trace)
        torch.cuda.synchronize()
        out[dc] = (xt.cpu().numpy(), trace.cpu().numpy())
        s.close()
    (xd, td), (xs, ts) = out[qg.QG_DC_DENSE], out[qg.QG_DC_SPARSE]
    assert np.max(np.abs(xs - xd)) <= 1e-9
    assert np.max(np.abs(ts - td) / np.abs(td)) <= 1e-10


def test_sparse_evaluation_is_bitwise_deterministic(qg):
    c = case_named("b1576")
    x = start(c, seed=8)
    for prec in (qg.QG_FP64, qg.QG_MIXED):
        s = qg.Solver(c, precision=prec, dc_solver=qg.QG_DC_SPARSE)
        xt = torch.tensor(x, dtype=s.dtype, device="cuda")
        o1, g1 = (t.clone() for t in s.eval_grad(xt))
        o2, g2 = (t.clone() for t in s.eval_grad(xt))
        assert torch.equal(o1, o2) and torch.equal(g1, g2)
        s.close()


def _peak_period(c):
    return int(np.argmax(c.load_p.sum(axis=1)))


@pytest.mark.parametrize("precision", [0, 1])
def test_dayahead_network_one_period_parity(qg, precision):
    """Full day-ahead network and all 2,000 outages at the peak-load period: objective, every
    term and the whole gradient against the oracle (sparse LU route)."""
    c0 = case_named("da")
    t = _peak_period(c0)
    c = synth.horizon_slice(c0, t, t + 1)
    x = start(c, seed=21)
    tol = TOL64
    if precision == 1:
        x, tol = as_f32(x), TOL32
    res = gpu_eval(qg, c, x, precision)  # QG_DC_AUTO: sparse above 4,096 buses
    check(res, oracle.evaluate(c, x, net=dayahead_net()), tol, c)


@pytest.mark.parametrize("precision", [0, 1])
def test_dayahead_full_horizon_sampled_period(qg, precision):
    """All 48 periods on the GPU; the oracle evaluates every non-contingency term and the
    contingency term of one sampled period, so the gradient rows of that period and every
    term but the contingency total are compared."""
    c = case_named("da")
    t = 31
    x = start(c, seed=22)
    tol = TOL64
    if precision == 1:
        x, tol = as_f32(x), TOL32
    obj, g, terms = gpu_eval(qg, c, x, precision)
    ref = oracle.evaluate(c, x, periods=[t], net=dayahead_net())
    assert np.all(np.isfinite(g))
    for k, name in enumerate(oracle.TERM_NAMES):
        if name != "zctg":
            assert abs(terms[0, k] - ref.terms[name]) <= tol * max(abs(ref.terms[name]), 1e-6 * abs(ref.obj)), name
    assert terms[0, oracle.TERM_NAMES.index("zctg")] >= ref.terms["zctg"]
    T, n, G = c.T, c.n_bus, c.n_gen
    rows = [("v", np.arange(t * n, (t + 1) * n)), ("theta", T * n + np.arange(t * n, (t + 1) * n))]
    rows += [(name, 2 * T * n + k * T * G + np.arange(t * G, (t + 1) * G)) for k, name in enumerate("pqr")]
    check_at(g, ref.grad, None, tol, f"period {t}", classes=rows)
