"""The bound test ahead of the contingency screen (qg_options.ctg_bound) changes no result.

A warp skips a chunk of periods only where max|L| max|f_k| over its columns is below every row's
clearance, which implies that the FP32 screen classifies none of its elements as a candidate (the
argument is at the kernel).  So with the bound test, and with the line-outage tile loaded up front
or on demand, the objective, the gradient, every objective term, the screening scores and a solve
trajectory are bitwise those of the element screen alone.  The cases cover both extremes: rt617 at
the copper-plate start (overloads present, some warp-chunks cleared), the same grid with ten times
its post-contingency ratings (no overload: every chunk cleared), and a random point far from
dispatch (hardly any cleared); plus a batch of uneven instances, phase shifters and a screening
handle."""
import dataclasses
import functools

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = (2, 3)  # QG_CTG_BOUND_EAGER, QG_CTG_BOUND_LAZY, each against QG_CTG_BOUND_OFF (1)


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
    return {"rt617": synth.rt617, "mid": synth.mid, "tiny": synth.tiny,
            "rt617_wide": lambda: dataclasses.replace(synth.rt617(), s_max_ctg=10.0 * synth.rt617().s_max_ctg),
            "mid_xf": lambda: synth.with_transformers(synth.mid(), 0.15, 5)}[name]()


def start(case, kind):
    if kind == "lp":
        return synth.lp_start(case)[0]
    if kind == "mo":
        from paper_2310_06650_gb300 import warmstart
        return warmstart.start_point(case)
    lo, hi = oracle.box(case)
    return np.clip(synth.random_point(case, 7), lo, hi)


def evaluate(qg, cases, x, precision, mode, **kw):
    s = qg.Solver(cases, precision=precision, ctg_bound=mode, **kw)
    try:
        xt = torch.tensor(x, dtype=s.dtype, device="cuda")
        obj, g = s.eval_grad(xt)
        torch.cuda.synchronize()
        return obj.cpu().numpy().copy(), g.cpu().numpy().copy(), s.breakdown()
    finally:
        s.close()


def assert_same(a, b):
    for u, v in zip(a, b):
        assert np.array_equal(u, v), np.max(np.abs(np.asarray(u, float) - np.asarray(v, float)))


@pytest.mark.parametrize("name,kind", [("rt617", "lp"), ("rt617_wide", "lp"), ("mid", "rand"),
                                       ("mid_xf", "mo"), ("tiny", "lp")])
@pytest.mark.parametrize("precision", [0, 1])
def test_bound_test_is_bitwise_neutral(qg, name, kind, precision):
    c = case_named(name)
    x = start(c, kind)
    ref = evaluate(qg, c, x, precision, 1)
    for mode in MODES:
        assert_same(evaluate(qg, c, x, precision, mode), ref)


def test_wide_ratings_have_no_contingency_overload(qg):
    """Every warp-chunk of the wide-rating case is cleared: the contingency term is its floor alone."""
    c = case_named("rt617_wide")
    x = start(c, "lp")
    ref = oracle.evaluate(c, x)
    assert ref.terms["zctg"] == pytest.approx(c.eps * c.c_s * c.beta * float(np.sum(c.dt)) * (c.n_branch - 1) * c.K,
                                              rel=1e-12)
    _, _, terms = evaluate(qg, c, x, 0, 3)
    assert terms[0, 7] == pytest.approx(ref.terms["zctg"], rel=1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_bound_test_batch(qg, precision):
    cases = [case_named("tiny"), case_named("mid"), synth.batch(per_shape=1)[0], case_named("rt617")]
    x = np.concatenate([start(c, "mo") for c in cases])
    ref = evaluate(qg, cases, x, precision, 1)
    for mode in MODES:
        assert_same(evaluate(qg, cases, x, precision, mode), ref)


def test_bound_test_screening_scores(qg):
    c = case_named("rt617")
    x = start(c, "lp")
    Ks = int(np.ceil(0.25 * c.K))
    sel = np.sort(np.random.default_rng(3).choice(c.K, Ks, replace=False))
    out = []
    for mode in (1,) + MODES:
        s = qg.Solver(c, precision=0, ctg_frac=0.25, ctg_bound=mode)
        qg.qg_ctg_select(s.h, 0, sel)
        obj, g = s.eval_grad(torch.tensor(x, dtype=s.dtype, device="cuda"))
        torch.cuda.synchronize()
        out.append((obj.cpu().numpy().copy(), g.cpu().numpy().copy(), qg.qg_ctg_scores(s.h, c.T * Ks)))
        s.close()
    for o in out[1:]:
        assert_same(o, out[0])


@pytest.mark.parametrize("precision", [0, 1])
def test_bound_test_solve_trajectory(qg, precision):
    c = case_named("rt617")
    x0 = start(c, "lp")
    xs = []
    for mode in (1,) + MODES:
        s = qg.Solver(c, precision=precision, ctg_bound=mode)
        x = torch.tensor(x0, dtype=s.dtype, device="cuda")
        qg.qg_solve(s.h, x, 20, 1e-3, 0.9, 0.999)
        torch.cuda.synchronize()
        xs.append(x.cpu().numpy().copy())
        s.close()
    for v in xs[1:]:
        assert np.array_equal(v, xs[0])


def test_bound_option_is_validated(qg):
    with pytest.raises(qg.QGError):
        qg.Solver(case_named("tiny"), precision=0, ctg_bound=4)


def test_resolved_path_and_launch_count(qg):
    """rt617 (small grid) resolves QG_CTG_BOUND_AUTO to no bound test; the on-demand path adds the
    clearance kernel to an evaluation's launches."""
    c = case_named("rt617")
    counts = {}
    for mode, path in ((0, 0), (1, 0), (2, 1), (3, 2)):
        s = qg.Solver(c, precision=1, ctg_bound=mode)
        assert qg.qg_ctg_path(s.h) == path
        counts[mode] = qg.qg_launches_per_eval(s.h)
        s.close()
    assert counts[0] == counts[1] == counts[2] == counts[3] - 1
