"""Device models through the C ABI against the FP64 oracle: bid-block costs (Example 3), consumers
(Example 4's balance sign, value subtracted from the objective) and relaxed on/off status with
startup / shutdown costs and u-scaled limits (Example 2); both DC solvers, both precisions, batched
with plain instances, and the graph-replayed Adam loop.

Tolerances as in the other parity tests: 1e-10 relative (FP64 path), 1e-4 (mixed path, with the
oracle evaluated at the same FP32-rounded point)."""
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


def devices(case, seed, commit=True):
    c = synth.with_block_bids(case, n_blocks=4, cons_frac=0.25, seed=seed)
    return synth.with_commitment(c, seed=seed) if commit else c


@functools.lru_cache(maxsize=None)
def case_named(name):
    return {"tiny": lambda: devices(synth.tiny(), 1),
            "tiny_xf": lambda: devices(synth.with_transformers(synth.tiny(), 0.3, 4), 2),
            "mid": lambda: devices(synth.mid(), 3),
            "mid_bids": lambda: devices(synth.mid(), 4, commit=False),
            "rt617": lambda: devices(synth.rt617(), 5)}[name]()


def start(case, seed=31):
    """Pmax-proportional dispatch (consumers too), flat voltage, perturbed inside the box; tau, phi
    and the on-status u drawn uniformly in their ranges."""
    x = case.flat_start(synth.proportional_dispatch(case)) + 0.02 * (synth.random_point(case, seed) - 0.5)
    otau, _ = case.offsets_xf()
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


@pytest.mark.parametrize("name", ["tiny", "tiny_xf", "mid", "mid_bids", "rt617"])
@pytest.mark.parametrize("dc", [1, 2])
def test_devices_fp64_parity(qg, name, dc):
    c = case_named(name)
    x = start(c)
    check(gpu_eval(qg, c, x, qg.QG_FP64, dc_solver=dc), oracle.evaluate(c, x), TOL64, c)


@pytest.mark.parametrize("name", ["mid", "rt617"])
@pytest.mark.parametrize("dc", [1, 2])
def test_devices_mixed_parity(qg, name, dc):
    c = case_named(name)
    x = as_f32(start(c))
    check(gpu_eval(qg, c, x, qg.QG_MIXED, dc_solver=dc), oracle.evaluate(c, x), TOL32, c)


def test_binary_status_and_block_edges(qg):
    """u at 0 and 1 with repeated values (no start or stop between equal periods) and dispatch at
    block edges and at 0: the derivative conventions (right derivative of the blocks, 0 for
    max(0, 0)) agree with the oracle's."""
    c = case_named("tiny")
    x = start(c, 5)
    rng = np.random.default_rng(2)
    u = (rng.uniform(size=(c.T, c.n_gen)) < 0.5).astype(float)
    u[1] = u[0]
    x[c.offset_u():] = u.ravel()
    o = c.offsets()
    p = x[o[2]:o[3]].reshape(c.T, c.n_gen)
    lo_edge = np.concatenate([np.zeros((c.n_gen, 1)), np.cumsum(c.blk_width, axis=1)[:, :-1]], axis=1)
    p[0] = lo_edge[:, 1]
    p[1] = 0.0
    x[o[2]:o[3]] = p.ravel()
    lo, hi = oracle.box(c)
    x = np.clip(x, lo, hi)
    check(gpu_eval(qg, c, x, qg.QG_FP64), oracle.evaluate(c, x), TOL64, c)


def test_devices_in_an_uneven_batch(qg):
    """Instances with consumers, bids and on-status beside plain ones in one handle."""
    cases = [case_named("tiny"), synth.tiny(), case_named("mid_bids"), case_named("tiny_xf"),
             synth.batch(per_shape=1)[0]]
    xs = [as_f32(start(c, 40 + i)) for i, c in enumerate(cases)]
    for prec, tol in ((qg.QG_FP64, TOL64), (qg.QG_MIXED, TOL32)):
        s = qg.Solver(cases, precision=prec)
        assert s.n_x == sum(c.n_x for c in cases)
        for b, c in enumerate(cases):
            first, n_x, off = qg.qg_layout(s.h, b)
            assert n_x == c.n_x and off[7] == c.offset_u()
        s.close()
        obj, g, _ = gpu_eval(qg, cases, np.concatenate(xs), prec)
        o = 0
        for b, (c, x) in enumerate(zip(cases, xs)):
            ref = oracle.evaluate(c, x)
            assert rel(obj[b], ref.obj) <= tol
            check_at(g[o:o + c.n_x], ref.grad, c, tol, f"instance {b}")
            o += c.n_x


@pytest.mark.parametrize("dc", [1, 2])
def test_devices_solve_trajectory_matches_oracle(qg, dc):
    """qg_solve (graph-replayed evaluation + fused Adam: p, q, r and u updated in the device stage
    with the on-status snapshot for the startup / shutdown terms) against the oracle's own loop."""
    c = case_named("tiny_xf")
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
    assert np.all(xg >= lo) and np.all(xg <= hi)
    ou = c.offset_u()
    assert np.max(np.abs(xg[ou:] - x0[ou:])) > 1e-3  # u moved
    s.close()
