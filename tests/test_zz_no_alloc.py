"""qg_eval_grad_noalloc: the evaluation for callers that cannot allocate device memory when they
evaluate (allocator locks, host callbacks, frozen memory pools).  Its work buffers come from the
library's static device scratch; its results must equal those of qg_eval_grad, call after call.

This file is collected last on purpose, so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""
import pytest

import synth

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


def start(c, seed):
    """The stored copper-plate start where the case has one, else the flat start, perturbed."""
    try:
        x0, _ = synth.lp_start(c)
    except FileNotFoundError:
        x0 = c.flat_start()
    return x0 + 0.01 * (synth.random_point(c, seed) - 0.5)


def noalloc(qg, s, x):
    """One qg_eval_grad_noalloc into NaN-filled outputs (nothing left from an earlier call can pass)."""
    obj = torch.full((s.n_inst,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((s.n_x,), float("nan"), dtype=s.dtype, device="cuda")
    qg.qg_eval_grad_noalloc(s.h, x, obj, g)
    torch.cuda.synchronize()
    return obj, g


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_eval_grad_twice(qg, precision):
    """The same kernels in the same order on the same data: bitwise the results of qg_eval_grad,
    on two calls in a row (the second starts from what the first left in the scratch)."""
    c = synth.rt617()
    s = qg.Solver(c, precision=precision)
    x = torch.tensor(start(c, 17), dtype=s.dtype, device="cuda")
    obj_ref, g_ref = (t.clone() for t in s.eval_grad(x))
    for _ in range(2):
        obj, g = noalloc(qg, s, x)
        assert torch.equal(obj, obj_ref)
        assert torch.equal(g, g_ref)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_alternating_handles_of_different_shapes(qg, precision):
    """Handles with different scratch layouts take turns on the one shared array; each call's result
    is still bitwise its own handle's qg_eval_grad, whatever the previous call left behind."""
    cases = [synth.tiny(), synth.rt617(), synth.mid()]
    solvers = [qg.Solver(c, precision=precision) for c in cases]
    xs = [torch.tensor(start(c, 30 + i), dtype=s.dtype, device="cuda") for i, (c, s) in enumerate(zip(cases, solvers))]
    refs = [tuple(t.clone() for t in s.eval_grad(x)) for s, x in zip(solvers, xs)]
    for k in (0, 1, 0, 2, 1, 2, 0):
        obj, g = noalloc(qg, solvers[k], xs[k])
        assert torch.equal(obj, refs[k][0]), k
        assert torch.equal(g, refs[k][1]), k
    for s in solvers:
        s.close()


def test_noalloc_allocates_nothing(qg):
    """After a first call (which looks up the scratch address), further calls change neither the
    device's free memory (cudaMemGetInfo) nor torch's allocator."""
    c = synth.rt617()
    s = qg.Solver(c, precision=1)
    x = torch.tensor(start(c, 5), dtype=s.dtype, device="cuda")
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(s.n_x, dtype=s.dtype, device="cuda")
    qg.qg_eval_grad_noalloc(s.h, x, obj, g)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        qg.qg_eval_grad_noalloc(s.h, x, obj, g)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    s.close()


def test_noalloc_rejects_handles_beyond_its_scratch(qg):
    cases = synth.batch(per_shape=1)  # one of each shape, incl. 1,576 buses x 48 periods
    s = qg.Solver(cases, precision=0)
    x = torch.zeros(s.n_x, dtype=torch.float64, device="cuda")
    obj = torch.zeros(len(cases), dtype=torch.float64, device="cuda")
    g = torch.zeros(s.n_x, dtype=torch.float64, device="cuda")
    with pytest.raises(qg.QGError) as ei:
        qg.qg_eval_grad_noalloc(s.h, x, obj, g)
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED and "scratch" in str(ei.value)
    s.close()


@pytest.mark.parametrize("kw,word", [(dict(ctg_frac=0.2), "screening"), (dict(dc_solver=2), "sparse")])
def test_noalloc_rejects_screening_and_sparse_handles(qg, kw, word):
    """Handles whose buffers are not carved from the scratch: contingency screening (its compacted
    line-outage block) and the sparse DC solver (its solve buffers)."""
    c = synth.tiny()
    s = qg.Solver(c, precision=0, **kw)
    x = torch.tensor(c.flat_start(), dtype=torch.float64, device="cuda")
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(s.n_x, dtype=torch.float64, device="cuda")
    with pytest.raises(qg.QGError) as ei:
        qg.qg_eval_grad_noalloc(s.h, x, obj, g)
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED and word in str(ei.value)
    s.close()
