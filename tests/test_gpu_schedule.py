"""Sec. II-F schedules on the GPU path: the graph-replayed Adam loop with a per-iteration step size,
soft-abs / soft-ReLU epsilon and homotopy scale (qg_solve_schedule), against the oracle's loop with
the same per-iteration values."""
import dataclasses

import numpy as np
import pytest

import oracle
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


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("mk,dc", [(synth.tiny, 1), (lambda: synth.with_transformers(synth.tiny(), 0.3, 4), 1),
                                   (synth.tiny, 2)])
def test_scheduled_solve_matches_oracle_loop(qg, mk, dc):
    c = mk()
    from oracle.copperplate import lambda_dispatch
    x0 = c.flat_start(lambda_dispatch(c))
    iters = 30
    sched = qg.qg_schedule(iters, 2e-3, 1e-5, 5e-2, 1e-4, 0.1, 1.0, 0.25)
    s = qg.Solver(c, precision=qg.QG_FP64, dc_solver=dc)
    xt = torch.tensor(x0, dtype=torch.float64, device="cuda")
    st = torch.tensor(sched, dtype=torch.float64, device="cuda")
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
    # two chunks of one run: the second continues the schedule and the trace
    qg.qg_solve_schedule(s.h, xt, 12, st, True, 0.9, 0.999, trace)
    qg.qg_solve_schedule(s.h, xt, iters - 12, st, False, 0.9, 0.999, trace)
    torch.cuda.synchronize()
    lo, hi = oracle.box(c)
    x, m, v = x0.copy(), np.zeros_like(x0), np.zeros_like(x0)
    tr = trace.cpu().numpy()
    for i in range(1, iters + 1):
        lr, eps, beta = sched[i - 1]
        ci = dataclasses.replace(c, eps=eps, beta=beta)
        ref = oracle.evaluate(ci, x)
        assert rel(tr[i - 1], ref.obj) <= 1e-9, (i, tr[i - 1], ref.obj)
        x, m, v = oracle.adam_step(x, m, v, ref.grad, i, lr, 0.9, 0.999, 1e-8, lo, hi)
    assert np.max(np.abs(xt.cpu().numpy() - x)) <= 1e-9
    # the handle's own options are untouched: a plain evaluation afterwards uses them
    obj, _ = s.eval_grad(xt)
    assert rel(obj.item(), oracle.evaluate(c, xt.cpu().numpy()).obj) <= 1e-10
    s.close()
