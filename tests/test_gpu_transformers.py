"""Transformers and phase shifters (tap ratio tau and phase shift phi as per-period variables)
through the C ABI, against the FP64 oracle: both DC solvers, both precisions, batched with
instances without transformers, and the graph-replayed Adam loop.

Tolerances as in the other parity tests: 1e-10 relative (FP64 path), 1e-4 (mixed path, with the
oracle evaluated at the same FP32-rounded point)."""
import functools

import numpy as np
import pytest

import oracle
import synth
from gradcheck import check_at
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
    return {"tiny": lambda: synth.with_transformers(synth.tiny(), 0.3, 4),
            "mid": lambda: synth.with_transformers(synth.mid(), 0.15, 5),
            "rt617": lambda: synth.with_transformers(synth.rt617(), 0.1, 6)}[name]()


def start(case, seed=31):
    """Merit-order dispatch, flat voltage, perturbed inside the box; tau and phi drawn in their ranges."""
    x = case.flat_start(lambda_dispatch(case)) + 0.02 * (synth.random_point(case, seed) - 0.5)
    otau, ophi = case.offsets_xf()
    xr = synth.random_point(case, seed + 1)
    x[otau:] = xr[otau:]
    lo, hi = oracle.box(case)
    return np.clip(x, lo, hi)


def as_f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grel(g, gr):
    return np.linalg.norm(g - gr) / np.linalg.norm(gr)


def gpu_eval(qg, cases, x, precision, **kw):
    s = qg.Solver(cases, precision=precision, **kw)
    xt = torch.tensor(x, dtype=s.dtype, device="cuda")
    obj, g = s.eval_grad(xt)
    torch.cuda.synchronize()
    out = (obj.cpu().numpy().copy(), g.double().cpu().numpy().copy(), s.breakdown())
    s.close()
    return out


def check(res, ref, tol, case):
    obj, g, terms = res
    assert rel(obj[0], ref.obj) <= tol, (obj[0], ref.obj)
    check_at(g, ref.grad, case, tol)
    for k, name in enumerate(oracle.TERM_NAMES):
        assert abs(terms[0, k] - ref.terms[name]) <= tol * max(abs(ref.terms[name]), 1e-6 * abs(ref.obj)), name


@pytest.mark.parametrize("name", ["tiny", "mid", "rt617"])
@pytest.mark.parametrize("dc", [1, 2])
def test_transformer_fp64_parity(qg, name, dc):
    c = case_named(name)
    x = start(c)
    check(gpu_eval(qg, c, x, qg.QG_FP64, dc_solver=dc), oracle.evaluate(c, x), TOL64, c)


@pytest.mark.parametrize("name", ["mid", "rt617"])
@pytest.mark.parametrize("dc", [1, 2])
def test_transformer_mixed_parity(qg, name, dc):
    c = case_named(name)
    x = as_f32(start(c))
    check(gpu_eval(qg, c, x, qg.QG_MIXED, dc_solver=dc), oracle.evaluate(c, x), TOL32, c)


def test_transformers_in_an_uneven_batch(qg):
    """Instances with and without transformers in one handle."""
    cases = [case_named("tiny"), synth.tiny(), case_named("mid"), synth.batch(per_shape=1)[0]]
    xs = [as_f32(start(c, 40 + i)) for i, c in enumerate(cases)]
    for prec, tol in ((qg.QG_FP64, TOL64), (qg.QG_MIXED, TOL32)):
        obj, g, _ = gpu_eval(qg, cases, np.concatenate(xs), prec)
        o = 0
        for b, (c, x) in enumerate(zip(cases, xs)):
            ref = oracle.evaluate(c, x)
            assert rel(obj[b], ref.obj) <= tol
            check_at(g[o:o + c.n_x], ref.grad, c, tol, f"instance {b}")
            o += c.n_x


@pytest.mark.parametrize("dc", [1, 2])
def test_transformer_solve_trajectory_matches_oracle(qg, dc):
    """qg_solve (graph-replayed evaluation + fused Adam on every block, tau and phi clipped to
    their ranges) against the oracle's own loop."""
    c = case_named("tiny")
    x0 = start(c, 7)
    iters = 40
    s = qg.Solver(c, precision=qg.QG_FP64, dc_solver=dc)
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
    otau, _ = c.offsets_xf()
    assert np.all(xg[otau:] >= lo[otau:]) and np.all(xg[otau:] <= hi[otau:])
    assert np.max(np.abs(xg[otau:] - x0[otau:])) > 1e-3  # tau and phi moved
    s.close()
