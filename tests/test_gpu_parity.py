"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: the FP64 path agrees with the oracle to 1e-10 relative on the objective and on every
objective term; the mixed path (FP32 flows / penalties / adjoints / Adam, double-FP32 DC solves,
FP64 objective accumulation and constraint residuals) to 1e-4.  Gradients are compared per variable
class and element by element (tests/gradcheck.py: class norms at 1e-10 / 1e-4, elements at
1e-10 / 1e-3 of their magnitude plus 0.1 of their class's largest entry).
"""
import numpy as np
import pytest

import oracle
import synth
from gradcheck import check64, check_prec, grad_errors
from oracle.copperplate import copper_plate

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


_CASES = {}


def case_named(name):
    if name not in _CASES:
        _CASES[name] = {"tiny": synth.tiny, "mid": synth.mid, "rt617": synth.rt617,
                        "b73": lambda: synth.batch(per_shape=1)[0]}[name]()
    return _CASES[name]


def point(case, kind):
    if kind == "lp":
        _, p, r = copper_plate(case)
        return case.flat_start(p, r)
    if kind == "lp_perturbed":
        _, p, r = copper_plate(case)
        x = case.flat_start(p, r) + 0.02 * (synth.random_point(case, 99) - 0.5)
        lo, hi = oracle.box(case)
        return np.clip(x, lo, hi)
    return synth.random_point(case, int(kind))


def gpu_eval(qg, cases, x, precision, lodf=0, **kw):
    s = qg.Solver(cases, precision=precision, lodf_dtype=lodf, **kw)
    xt = torch.tensor(x, dtype=s.dtype, device="cuda")
    obj, g = s.eval_grad(xt)
    torch.cuda.synchronize()
    out = (obj.cpu().numpy().copy(), g.double().cpu().numpy().copy(), s.breakdown())
    s.close()
    return out


def as_f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grel(g, gr):
    return np.linalg.norm(g - gr) / np.linalg.norm(gr)


def check(res, ref, tol, case, precision):
    obj, g, terms = res
    assert rel(obj[0], ref.obj) <= tol, (obj[0], ref.obj)
    check_prec(g, ref.grad, case, precision)
    for k, name in enumerate(oracle.TERM_NAMES):
        assert abs(terms[0, k] - ref.terms[name]) <= tol * max(abs(ref.terms[name]), 1e-6 * abs(ref.obj)), name


@pytest.mark.parametrize("name,kind", [("tiny", "1"), ("tiny", "lp"), ("mid", "2"), ("mid", "lp_perturbed"),
                                       ("rt617", "3"), ("rt617", "lp"), ("rt617", "lp_perturbed")])
def test_fp64_parity(qg, name, kind):
    c = case_named(name)
    x = point(c, kind)
    check(gpu_eval(qg, c, x, qg.QG_FP64), oracle.evaluate(c, x), TOL64, c, qg.QG_FP64)


@pytest.mark.parametrize("name,kind", [("tiny", "1"), ("mid", "lp_perturbed"), ("rt617", "lp"),
                                       ("rt617", "lp_perturbed")])
def test_mixed_parity(qg, name, kind):
    """The mixed path keeps x in FP32, so the oracle is evaluated at the same FP32-rounded point."""
    c = case_named(name)
    x = as_f32(point(c, kind))
    check(gpu_eval(qg, c, x, qg.QG_MIXED), oracle.evaluate(c, x), TOL32, c, qg.QG_MIXED)


def test_eps_zero_scoring_parity(qg):
    """The metric scores points with the hard abs / ReLU (eps = 0)."""
    c = case_named("mid")
    x = point(c, "lp_perturbed")
    res = gpu_eval(qg, c, x, qg.QG_FP64, eps=0.0)
    ref = oracle.evaluate(c, x, eps=0.0)
    assert rel(res[0][0], ref.obj) <= TOL64
    check64(res[1], ref.grad, c)


def test_ragged_batch_parity(qg):
    """Uneven instances in one handle: every instance matches its own oracle evaluation."""
    cases = [case_named("tiny"), case_named("mid"), case_named("b73"), synth.tiny(seed=5)]
    xs = [as_f32(point(c, str(10 + i))) for i, c in enumerate(cases)]
    for prec, tol in ((qg.QG_FP64, TOL64), (qg.QG_MIXED, TOL32)):
        obj, g, terms = gpu_eval(qg, cases, np.concatenate(xs), prec)
        o = 0
        for b, (c, x) in enumerate(zip(cases, xs)):
            ref = oracle.evaluate(c, x)
            assert rel(obj[b], ref.obj) <= tol
            check_prec(g[o:o + c.n_x], ref.grad, c, prec, f"instance {b}")
            o += c.n_x


def test_evaluation_is_bitwise_deterministic(qg):
    c = case_named("rt617")
    x = point(c, "lp_perturbed")
    for prec in (qg.QG_FP64, qg.QG_MIXED):
        s = qg.Solver(c, precision=prec)
        xt = torch.tensor(x, dtype=s.dtype, device="cuda")
        o1, g1 = (t.clone() for t in s.eval_grad(xt))
        o2, g2 = (t.clone() for t in s.eval_grad(xt))
        assert torch.equal(o1, o2) and torch.equal(g1, g2)
        s.close()


def test_host_entry_matches_device_entry(qg):
    c = case_named("mid")
    x = point(c, "lp_perturbed")
    for prec in (qg.QG_FP64, qg.QG_MIXED):
        s = qg.Solver(c, precision=prec)
        obj_h = np.zeros(1)
        g_h = np.zeros(c.n_x)
        qg.qg_eval_grad_host(s.h, np.ascontiguousarray(x), obj_h, g_h)
        xt = torch.tensor(x, dtype=s.dtype, device="cuda")
        obj, g = s.eval_grad(xt)
        torch.cuda.synchronize()
        assert obj_h[0] == obj.item()
        assert np.array_equal(g_h, g.double().cpu().numpy())
        s.close()


def test_host_entry_with_pinned_buffers_replays_a_graph(qg):
    """Page-locked host buffers take the cached-graph route: the same results as the device entry,
    call after call, with new contents in the same buffers and with other buffers."""
    c = case_named("mid")
    for prec in (qg.QG_FP64, qg.QG_MIXED):
        s = qg.Solver(c, precision=prec)
        xs = [point(c, "lp_perturbed"), point(c, "3")]
        bufs = [(torch.zeros(c.n_x, dtype=torch.float64).pin_memory(), torch.zeros(1, dtype=torch.float64).pin_memory(),
                 torch.zeros(c.n_x, dtype=torch.float64).pin_memory()) for _ in range(2)]
        for k, x in enumerate(xs + xs):
            xb, ob, gb = bufs[k // 2 % 2]
            xb.copy_(torch.from_numpy(x))
            qg.qg_eval_grad_host(s.h, xb.numpy(), ob.numpy(), gb.numpy())
            obj, g = s.eval_grad(torch.tensor(x, dtype=s.dtype, device="cuda"))
            torch.cuda.synchronize()
            assert ob.item() == obj.item(), k
            assert np.array_equal(gb.numpy(), g.double().cpu().numpy()), k
        s.close()


def test_host_entry_reports_a_nonfinite_objective(qg):
    """A NaN in x makes the objective NaN: the host entry writes its outputs, returns
    QG_ERR_NONFINITE, and the handle evaluates the next finite point normally."""
    c = case_named("tiny")
    for prec in (qg.QG_FP64, qg.QG_MIXED):
        s = qg.Solver(c, precision=prec)
        x = point(c, "1")
        bad = x.copy()
        bad[c.offsets()[0] + 3] = np.nan
        obj, g = np.zeros(1), np.zeros(c.n_x)
        with pytest.raises(qg.QGError) as ei:
            qg.qg_eval_grad_host(s.h, bad, obj, g)
        assert ei.value.code == qg.QG_ERR_NONFINITE and "not finite" in str(ei.value)
        assert np.isnan(obj[0])
        qg.qg_eval_grad_host(s.h, x, obj, g)
        ref = oracle.evaluate(c, x if prec == qg.QG_FP64 else as_f32(x))
        assert rel(obj[0], ref.obj) <= (TOL64 if prec == qg.QG_FP64 else TOL32)
        s.close()


def test_adam_step_parity(qg):
    c = case_named("mid")
    x = point(c, "lp_perturbed")
    s = qg.Solver(c, precision=qg.QG_FP64)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    m = torch.zeros_like(xt)
    v = torch.zeros_like(xt)
    lo, hi = oracle.box(c)
    xr, mr, vr = x.copy(), np.zeros_like(x), np.zeros_like(x)
    for i in range(1, 6):
        _, g = s.eval_grad(xt)
        gr = g.cpu().numpy().copy()
        qg.qg_adam_step(s.h, xt, m, v, 1e-3, 0.9, 0.999)
        xr, mr, vr = oracle.adam_step(xr, mr, vr, gr, i, 1e-3, 0.9, 0.999, 1e-8, lo, hi)
        torch.cuda.synchronize()
        assert np.max(np.abs(xt.cpu().numpy() - xr)) <= 1e-14
        assert np.max(np.abs(m.cpu().numpy() - mr)) <= 1e-12 * np.abs(mr).max()
    assert qg.qg_get_step(s.h) == 5
    s.close()


def test_solve_trajectory_matches_oracle(qg):
    """qg_solve (graph-replayed eval + Adam) against the oracle's own loop, per iterate."""
    c = case_named("tiny")
    x0 = point(c, "lp")
    iters = 60
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
    assert np.max(np.abs(xt.cpu().numpy() - x)) <= 1e-9
    s.close()


def test_tiny_config_500_iteration_trajectory(qg):
    """The tiny configuration as specified: 500 projected-Adam iterations (lr 1e-3) from the
    copper-plate dispatch with flat voltage.  Every iterate of the GPU run is checked against the
    oracle at the GPU's own point (objective, gradient, and the Adam step from the GPU's moments):
    two independent 500-step runs drift apart through rounding (Adam's normalized steps amplify the
    sign of near-zero gradients), so the comparison is per step.  The graph-replayed loop with the
    fused update (qg_solve) then follows the step-by-step run until the same drift sets in."""
    c = case_named("tiny")
    x0 = point(c, "lp")
    iters = 500
    lo, hi = oracle.box(c)
    s = qg.Solver(c, precision=qg.QG_FP64)
    xt = torch.tensor(x0, dtype=torch.float64, device="cuda")
    m = torch.zeros_like(xt)
    v = torch.zeros_like(xt)
    objs = []
    for i in range(1, iters + 1):
        obj, g = s.eval_grad(xt)
        xn, gn = xt.cpu().numpy().copy(), g.cpu().numpy().copy()
        mn, vn = m.cpu().numpy().copy(), v.cpu().numpy().copy()
        ref = oracle.evaluate(c, xn)
        objs.append(obj[0].item())
        assert rel(objs[-1], ref.obj) <= 1e-10, i
        check64(gn, ref.grad, c, f"iteration {i}")
        qg.qg_adam_step(s.h, xt, m, v, 1e-3, 0.9, 0.999)
        xr, _, _ = oracle.adam_step(xn, mn, vn, gn, i, 1e-3, 0.9, 0.999, 1e-8, lo, hi)
        assert np.max(np.abs(xt.cpu().numpy() - xr)) <= 1e-13, i
    assert objs[-1] < 0.5 * objs[0]  # the run makes progress
    s2 = qg.Solver(c, precision=qg.QG_FP64)
    xs = torch.tensor(x0, dtype=torch.float64, device="cuda")
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
    qg.qg_solve(s2.h, xs, iters, 1e-3, 0.9, 0.999, trace)
    torch.cuda.synchronize()
    tr = trace.cpu().numpy()
    dev = np.array([rel(a, b) for a, b in zip(tr, objs)])
    # the fused and the step-by-step runs round differently (not bitwise equal): they agree closely
    # until the amplification described above sets in (measured: first gap above 1e-12 at iteration
    # 78, 2.9e-9 by iteration 100, 10% at most over 500), and both make the same progress
    assert dev[:60].max() <= 1e-9
    assert dev.max() <= 0.25 and tr[-1] < 0.5 * tr[0]
    s.close()
    s2.close()


def test_unrolled_solve_graph_equals_single_iterations(qg):
    """Long solves replay a graph of several iterations; the result is bitwise that of replaying the
    one-iteration graph as often (the same kernels in the same order)."""
    c = case_named("mid")
    x0 = point(c, "lp_perturbed")
    iters = 19
    out = []
    for chunk in (iters, 1):
        s = qg.Solver(c, precision=qg.QG_MIXED)
        xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
        if chunk == iters:
            qg.qg_solve(s.h, xt, iters, 1e-3, 0.9, 0.999)
        else:
            for _ in range(iters):
                qg.qg_solve(s.h, xt, 1, 1e-3, 0.9, 0.999)
        torch.cuda.synchronize()
        out.append((xt.cpu().clone(), qg.qg_get_step(s.h)))
        s.close()
    assert out[0][1] == out[1][1] == iters
    assert torch.equal(out[0][0], out[1][0])


def test_batch_config_parity(qg):
    """The 32-instance uneven batch (73/200/617/1576 buses, 12/18/24/48 periods) in one handle;
    every instance checked against the oracle on objective, terms and gradient, in both paths."""
    from oracle.copperplate import lambda_dispatch
    cases = synth.batch()
    xs = [as_f32(c.flat_start(lambda_dispatch(c))) for c in cases]
    X = np.concatenate(xs)
    offs = np.cumsum([0] + [c.n_x for c in cases])
    refs = [oracle.evaluate(c, x) for c, x in zip(cases, xs)]
    for prec, tol in ((qg.QG_FP64, TOL64), (qg.QG_MIXED, TOL32)):
        obj, g, terms = gpu_eval(qg, cases, X, prec)
        assert np.all(np.isfinite(obj)) and np.all(np.isfinite(g))
        for b, (c, ref) in enumerate(zip(cases, refs)):
            assert rel(obj[b], ref.obj) <= tol, (b, obj[b], ref.obj)
            check_prec(g[offs[b]:offs[b + 1]], ref.grad, c, prec, f"instance {b}")
            for k, name in enumerate(oracle.TERM_NAMES):
                assert abs(terms[b, k] - ref.terms[name]) <= tol * max(abs(ref.terms[name]), 1e-6 * abs(ref.obj)), (b, name)


def test_lodf_low_precision_gate(qg, capsys):
    """BF16 storage of the line-outage block only where the mixed-path error stays under 1e-4:
    the hi+lo BF16 pair (about 2^-17 relative per entry) passes the gate at the copper-plate start;
    a single BF16 (2^-9) is reported, and the library keeps FP32 as its default."""
    c = case_named("rt617")
    x = as_f32(point(c, "lp_perturbed"))
    ref = oracle.evaluate(c, x)
    errs = {}
    for name, dt in (("f32", qg.QG_LODF_F32), ("bf16x2", qg.QG_LODF_BF16X2), ("bf16", qg.QG_LODF_BF16)):
        obj, g, _ = gpu_eval(qg, c, x, qg.QG_MIXED, lodf=dt)
        cls = grad_errors(g, ref.grad, c)
        errs[name] = (rel(obj[0], ref.obj), grel(g, ref.grad), max(e[0] for e in cls.values()),
                      max(e[1] for e in cls.values()))
    with capsys.disabled():
        print("\nLODF storage vs FP64 oracle (obj rel, grad rel, worst class rel, worst element):",
              {k: tuple(f"{v:.2e}" for v in e) for k, e in errs.items()})
    for name in ("f32", "bf16x2"):
        assert max(errs[name][:3]) <= TOL32, name
        assert errs[name][3] <= 10 * TOL32, name
    assert qg.qg_default_options().lodf_dtype == qg.QG_LODF_F32
