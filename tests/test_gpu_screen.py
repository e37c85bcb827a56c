"""The FP64 path's overload classification is FP64's, at an element built to sit on the edge.

On the phase-shifter ring of tests/screen_model.py, the monitored branch's post-contingency flow
cancels ~6,600 pu of loop flow down to 0.47 pu, and its rating is set so that the element is
overloaded in FP64 while its FP32 value (off by 4e-4 pu) is under the limit by more than a fixed
1e-4 s_ctg^2 margin.  The GPU's FP64 path must still count it.

Tolerance: at a 14,000 : 1 cancellation FP64 itself holds the element only to ~1e-12 relative, so
two exact FP64 formulations disagree well above 1e-10 (the oracle's rank-1 route against its
brute-force re-solve: 3e-10 on the contingency term, 3e-8 on the dispatch gradient).  The GPU is
held to 10 times that disagreement, and the test checks that leaving the element out would miss
by over a thousand times more."""
import numpy as np
import pytest

import oracle
from gradcheck import class_slices, grad_errors
from screen_model import dropped_by_fixed_margin

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


@pytest.mark.parametrize("dc", [1, 2])
def test_fp64_path_keeps_a_near_cancelling_overload(qg, dc):
    import dataclasses
    c, x, kk, e = dropped_by_fixed_margin()
    ref = oracle.evaluate(c, x)
    alt = oracle.evaluate(c, x, mode="brute")
    without = oracle.evaluate(dataclasses.replace(c, s_max_ctg=np.full(c.n_branch, 1e6)), x)
    zc = oracle.TERM_NAMES.index("zctg")
    tol_z = max(1e-10, 10 * abs(alt.terms["zctg"] - ref.terms["zctg"]) / ref.terms["zctg"])
    cls = grad_errors(alt.grad, ref.grad, c)
    tol_g = {k: max(1e-10, 10 * v[0]) for k, v in cls.items()}
    # leaving the edge element out moves the term and the gradient by far more than the tolerance
    assert abs(without.terms["zctg"] - ref.terms["zctg"]) > 1e3 * tol_z * ref.terms["zctg"]
    s = qg.Solver(c, precision=qg.QG_FP64, dc_solver=dc)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    obj, g = s.eval_grad(xt)
    torch.cuda.synchronize()
    terms = s.breakdown()
    gn = g.cpu().numpy()
    assert abs(obj.item() - ref.obj) <= 1e-10 * abs(ref.obj)
    assert abs(terms[0, zc] - ref.terms["zctg"]) <= tol_z * ref.terms["zctg"]
    for name, sl in class_slices(c):
        nr = np.linalg.norm(ref.grad[sl])
        assert np.linalg.norm(gn[sl] - ref.grad[sl]) <= tol_g[name] * nr, name
        if name == "p":  # the dispatch gradient carries the element's adjoint
            assert np.linalg.norm(without.grad[sl] - ref.grad[sl]) > 1e3 * tol_g[name] * nr
    s.close()
