"""The contingency-block shape autotuner (qg_autotune): it re-plans the handle, keeps a valid shape,
and leaves results equal to those of the heuristic shape up to the order of the outage sums; the
re-planned handle still runs the graph-replayed loop, screening and batches."""
import numpy as np
import pytest

import oracle
import synth
from gradcheck import check_at, check_grad

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import qg as mod
    return mod


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grel(g, gr):
    return np.linalg.norm(g - gr) / np.linalg.norm(gr)


def evaluate(s, x):
    obj, g = s.eval_grad(x)
    torch.cuda.synchronize()
    return obj.cpu().numpy().copy(), g.double().cpu().numpy().copy()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_autotune_keeps_parity_on_rt617(qg, precision, tol):
    c = synth.rt617()
    x0, _ = synth.lp_start(c)
    x0 = x0 + 0.01 * (synth.random_point(c, 3) - 0.5)
    if precision == 1:
        x0 = x0.astype(np.float32).astype(np.float64)
    s = qg.Solver(c, precision=precision)
    x = torch.tensor(x0, dtype=s.dtype, device="cuda")
    o1, g1 = evaluate(s, x)
    shape = qg.qg_autotune(s.h, x, 3, cold=(precision == 1))
    assert 1 <= shape[0] <= c.T and 1 <= shape[1] <= -(-c.n_branch // 64)
    assert tuple(qg.qg_tile_shape(s.h, 0)) == tuple(shape)
    o2, g2 = evaluate(s, x)
    assert rel(o2[0], o1[0]) <= (1e-13 if precision == 0 else 1e-6)
    assert grel(g2, g1) <= (1e-13 if precision == 0 else 1e-6)
    ref = oracle.evaluate(c, x0)
    assert rel(o2[0], ref.obj) <= tol
    check_at(g2, ref.grad, c, tol)
    s.close()


def test_autotuned_batch_and_solve_loop(qg):
    """An uneven batch, autotuned, against the oracle; then qg_solve on the re-planned handle against a
    handle that kept the heuristic shape."""
    cases = [synth.tiny(), synth.batch(per_shape=1)[0], synth.with_transformers(synth.mid(), 0.15, 5)]
    xs = [np.clip(c.flat_start() + 0.02 * (synth.random_point(c, 50 + i) - 0.5), *oracle.box(c))
          for i, c in enumerate(cases)]
    x0 = np.concatenate(xs)
    s = qg.Solver(cases, precision=0)
    x = torch.tensor(x0, dtype=torch.float64, device="cuda")
    qg.qg_autotune(s.h, x, 2)
    obj, g = evaluate(s, x)
    o = 0
    for b, (c, xc) in enumerate(zip(cases, xs)):
        ref = oracle.evaluate(c, xc)
        assert rel(obj[b], ref.obj) <= 1e-10
        check_at(g[o:o + c.n_x], ref.grad, c, 1e-10, f"instance {b}")
        o += c.n_x
    s2 = qg.Solver(cases, precision=0)
    xa, xb = x.clone(), x.clone()
    qg.qg_solve(s.h, xa, 5, 1e-3, 0.9, 0.999)
    qg.qg_solve(s2.h, xb, 5, 1e-3, 0.9, 0.999)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(xa - xb)).item() <= 1e-9  # the shapes differ only in summation order
    s.close()
    s2.close()


def test_autotune_with_screening(qg):
    c = synth.mid()
    x0 = np.clip(c.flat_start() + 0.02 * (synth.random_point(c, 9) - 0.5), *oracle.box(c))
    s = qg.Solver(c, precision=0, ctg_frac=0.3)
    Ks = int(np.ceil(0.3 * c.K))
    sel = np.sort(np.random.default_rng(1).choice(c.K, Ks, replace=False)).astype(np.int32)
    qg.qg_ctg_select(s.h, 0, sel)
    x = torch.tensor(x0, dtype=torch.float64, device="cuda")
    qg.qg_autotune(s.h, x, 2)
    obj, g = evaluate(s, x)
    import dataclasses
    ref = oracle.evaluate(dataclasses.replace(c, ctg=c.ctg[sel]), x0)
    assert rel(obj[0], ref.obj) <= 1e-10
    check_at(g, ref.grad, c, 1e-10)
    s.close()


def test_a_later_handle_with_smaller_blocks_leaves_an_earlier_one_working(qg):
    """The contingency kernel's shared-memory limit is process-wide: a handle created later with a
    smaller period chunk must not lower it under an existing handle's need."""
    big = synth.batch(per_shape=1)[3]  # 1,576 buses x 48 periods
    s1 = qg.Solver(big, precision=1)
    x1 = torch.tensor(big.flat_start(), dtype=torch.float32, device="cuda")
    qg.qg_autotune(s1.h, x1, 1)  # may pick a long period chunk
    small = synth.tiny()
    s2 = qg.Solver(small, precision=1)
    o, g = evaluate(s1, x1)
    ref = oracle.evaluate(big, big.flat_start().astype(np.float32).astype(np.float64))
    assert rel(o[0], ref.obj) <= 1e-4
    s1.close()
    s2.close()
