"""Contingency screening (Alg. 2) through the C ABI: a screening handle evaluates a selected subset
of the outages through a compacted line-outage block; its objective, gradient and per-outage scores
equal the oracle's on the case restricted to that subset, before and after the subset changes, in
both precisions and in a batch; the running-list policy drives a solve."""
import dataclasses

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


def start(case, seed=51):
    x = case.flat_start(lambda_dispatch(case)) + 0.02 * (synth.random_point(case, seed) - 0.5)
    lo, hi = oracle.box(case)
    return np.clip(x, lo, hi)


def as_f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grel(g, gr):
    return np.linalg.norm(g - gr) / np.linalg.norm(gr)


def subset(case, sel):
    return dataclasses.replace(case, ctg=case.ctg[np.asarray(sel)])


def floor_per_pair(case):
    """Soft-ReLU floor of one (period, outage) score: d_t c_s beta eps for every monitored branch."""
    return case.dt[:, None] * case.c_s * case.beta * case.eps * (case.n_branch - 1)


@pytest.mark.parametrize("name,prec", [("mid", 0), ("rt617", 0), ("rt617", 1)])
def test_screened_evaluation_matches_the_oracle_on_the_subset(qg, name, prec):
    c = {"mid": synth.mid, "rt617": synth.rt617}[name]()
    x = start(c)
    tol = TOL64
    if prec == 1:
        x, tol = as_f32(x), TOL32
    s = qg.Solver(c, precision=prec, ctg_frac=0.25)
    Ks = int(np.ceil(0.25 * c.K))
    rng = np.random.default_rng(3)
    for sel in (np.arange(Ks), np.sort(rng.choice(c.K, Ks, replace=False))):
        if sel[0] != 0 or not np.array_equal(sel, np.arange(Ks)):
            qg.qg_ctg_select(s.h, 0, sel)
        xt = torch.tensor(x, dtype=s.dtype, device="cuda")
        obj, g = s.eval_grad(xt)
        torch.cuda.synchronize()
        ref = oracle.evaluate(subset(c, sel), x)
        assert rel(obj.item(), ref.obj) <= tol, (obj.item(), ref.obj)
        check_at(g.double().cpu().numpy(), ref.grad, c, tol)
        terms = s.breakdown()
        assert abs(terms[0, 7] - ref.terms["zctg"]) <= tol * abs(ref.terms["zctg"])
        z = qg.qg_ctg_scores(s.h, c.T * Ks).reshape(c.T, Ks)
        zr = ref.z_ctg - floor_per_pair(c)
        assert np.max(np.abs(z - zr)) <= max(tol, 1e-9) * np.abs(zr).max() + 1e-9, np.max(np.abs(z - zr))
        assert np.abs(zr).max() > 0  # overloaded outages in the subset
    s.close()


def test_full_selection_equals_the_unscreened_handle(qg):
    c = synth.mid()
    x = start(c)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    a = qg.Solver(c, precision=0)
    b = qg.Solver(c, precision=0, ctg_frac=0.999)  # Ks = K
    oa, ga = (t.clone() for t in a.eval_grad(xt))
    ob, gb = (t.clone() for t in b.eval_grad(xt))
    assert rel(ob.item(), oa.item()) <= 1e-12
    check_grad(gb.cpu().numpy(), ga.cpu().numpy(), c, 1e-12, 1e-12)
    a.close()
    b.close()


def test_screened_batch(qg):
    cases = [synth.tiny(), synth.mid()]
    xs = [start(c, 60 + i) for i, c in enumerate(cases)]
    s = qg.Solver(cases, precision=0, ctg_frac=0.5)
    sels = []
    for i, c in enumerate(cases):
        Ks = int(np.ceil(0.5 * c.K))
        sel = np.sort(np.random.default_rng(i).choice(c.K, Ks, replace=False))
        qg.qg_ctg_select(s.h, i, sel)
        sels.append(sel)
    xt = torch.tensor(np.concatenate(xs), dtype=torch.float64, device="cuda")
    obj, g = s.eval_grad(xt)
    torch.cuda.synchronize()
    gn = g.cpu().numpy()
    o = 0
    for b, (c, x, sel) in enumerate(zip(cases, xs, sels)):
        ref = oracle.evaluate(subset(c, sel), x)
        assert rel(obj[b].item(), ref.obj) <= TOL64
        check_at(gn[o:o + c.n_x], ref.grad, c, TOL64, f"instance {b}")
        o += c.n_x
    s.close()


def test_subset_change_between_graph_replays(qg):
    """qg_solve keeps its captured graph across qg_ctg_select; the trajectory follows the oracle
    with the subset switched at the same iteration."""
    c = synth.tiny()
    x0 = start(c, 7)
    s = qg.Solver(c, precision=0, ctg_frac=0.5)
    Ks = int(np.ceil(0.5 * c.K))
    sel2 = np.arange(c.K - Ks, c.K)
    xt = torch.tensor(x0, dtype=torch.float64, device="cuda")
    qg.qg_solve(s.h, xt, 10, 1e-3, 0.9, 0.999)
    qg.qg_ctg_select(s.h, 0, sel2)
    qg.qg_solve(s.h, xt, 10, 1e-3, 0.9, 0.999)
    torch.cuda.synchronize()
    lo, hi = oracle.box(c)
    x, m, v = x0.copy(), np.zeros_like(x0), np.zeros_like(x0)
    for i in range(1, 21):
        cs = subset(c, np.arange(Ks) if i <= 10 else sel2)
        x, m, v = oracle.adam_step(x, m, v, oracle.evaluate(cs, x).grad, i, 1e-3, 0.9, 0.999, 1e-8, lo, hi)
    assert np.max(np.abs(xt.cpu().numpy() - x)) <= 1e-9
    s.close()


def test_selection_is_validated(qg):
    c = synth.tiny()
    s = qg.Solver(c, precision=0, ctg_frac=0.5)
    Ks = int(np.ceil(0.5 * c.K))
    with pytest.raises(qg.QGError):
        qg.qg_ctg_select(s.h, 0, np.arange(Ks - 1))
    dup = np.arange(Ks); dup[1] = dup[0]
    with pytest.raises(qg.QGError):
        qg.qg_ctg_select(s.h, 0, dup)
    s.close()
    plain = qg.Solver(c, precision=0)
    with pytest.raises(qg.QGError) as ei:
        qg.qg_ctg_select(plain.h, 0, np.arange(Ks))
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED
    plain.close()


def test_running_list_screened_solve_tracks_the_full_solve(qg):
    """Alg. 2 on rt617: half the outages per iteration (the worst-scoring half of the subset plus a
    random draw), re-selected every 25 iterations; after 500 iterations the full objective is close
    to that of the unscreened solve."""
    from paper_2310_06650_gb300 import screening
    c = synth.rt617()
    x0, _ = synth.lp_start(c)
    full = qg.Solver(c, precision=1)
    xa = torch.tensor(x0, dtype=torch.float32, device="cuda")
    qg.qg_solve(full.h, xa, 500, 1e-3, 0.9, 0.999)
    scr = qg.Solver(c, precision=1, ctg_frac=0.5)
    xb = torch.tensor(x0, dtype=torch.float32, device="cuda")
    screening.screened_solve(scr, xb, 500, 25, top_frac=0.5, seed=1)
    oa, _ = full.eval_grad(xa)
    ob, _ = full.eval_grad(xb)  # score both with every outage
    torch.cuda.synchronize()
    assert ob.item() <= 1.10 * oa.item(), (ob.item(), oa.item())
    full.close()
    scr.close()
