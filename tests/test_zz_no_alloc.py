"""qg_eval_grad_noalloc: the evaluation for callers that cannot allocate device memory when they
evaluate (allocator locks, host callbacks, frozen memory pools).  Its work buffers come from the
library's static device scratch; its results must equal those of qg_eval_grad, call after call.

This file is collected last on purpose, so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {0: 1e-10, 1: 1e-4}  # the parity tolerances of the FP64 and mixed paths


@pytest.fixture(scope="module")
def qg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import qg as mod
    return mod


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_eval_grad_twice(qg, precision):
    c = synth.rt617()
    x0, _ = synth.lp_start(c)
    x0 = x0 + 0.01 * (synth.random_point(c, 17) - 0.5)
    s = qg.Solver(c, precision=precision)
    x = torch.tensor(x0, dtype=s.dtype, device="cuda")
    obj_ref, g_ref = (t.clone() for t in s.eval_grad(x))
    for _ in range(2):
        obj = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full_like(g_ref, float("nan"))
        qg.qg_eval_grad_noalloc(s.h, x, obj, g)
        torch.cuda.synchronize()
        tol = TOL[precision]
        assert abs(obj.item() - obj_ref.item()) <= tol * abs(obj_ref.item())
        gn, gr = g.double().cpu().numpy(), g_ref.double().cpu().numpy()
        assert np.all(np.isfinite(gn))
        assert np.linalg.norm(gn - gr) <= tol * np.linalg.norm(gr)
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
