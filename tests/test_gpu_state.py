"""Checkpoint and resume of a solve (qg_get_state / qg_set_state).

Alg. 3's iteration carries (x, m, v, i); a scheduled run (Sec. II-F) also its position in the
schedule, contingency screening (Alg. 2) the outage selection, batch rounding (Alg. 1) the fixed
pairs and their clip box.  A run of 2N iterations straight through and a run of N iterations,
saved, restored into a new handle built from the same inputs and continued for N more must give
bitwise the same iterates (the same kernels in the same order)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 13  # one graph of 8 fused iterations plus 5 single ones per half


@pytest.fixture(scope="module")
def qg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import qg as mod
    return mod


def start(c, seed=3):
    x = c.flat_start(synth.proportional_dispatch(c)) + 0.02 * (synth.random_point(c, seed) - 0.5)
    return np.clip(x, *oracle.box(c))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["mid", "rt617"])
def test_solve_resumes_bitwise(qg, precision, name):
    c = {"mid": synth.mid, "rt617": synth.rt617}[name]()
    x0 = start(c)
    a = qg.Solver(c, precision=precision)
    xa = torch.tensor(x0, dtype=a.dtype, device="cuda")
    qg.qg_solve(a.h, xa, 2 * N, 1e-3, 0.9, 0.999)
    b = qg.Solver(c, precision=precision)
    xb = torch.tensor(x0, dtype=b.dtype, device="cuda")
    qg.qg_solve(b.h, xb, N, 1e-3, 0.9, 0.999)
    blob = qg.qg_get_state(b.h)
    assert len(blob) == qg.qg_state_size(b.h)
    xsave = xb.clone()
    b.close()
    r = qg.Solver(c, precision=precision)
    qg.qg_set_state(r.h, blob)
    assert qg.qg_get_step(r.h) == N
    qg.qg_solve(r.h, xsave, N, 1e-3, 0.9, 0.999)
    torch.cuda.synchronize()
    assert qg.qg_get_step(r.h) == qg.qg_get_step(a.h) == 2 * N
    assert torch.equal(xsave, xa)
    assert qg.qg_get_state(r.h) == qg.qg_get_state(a.h)  # moments and counters too
    assert not torch.equal(xa, torch.tensor(x0, dtype=a.dtype, device="cuda"))
    a.close()
    r.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_scheduled_solve_resumes_at_its_schedule_position(qg, precision):
    """A Sec. II-F run driven in two chunks across a checkpoint: the second chunk continues at row N
    of the schedule (lr, eps, beta) and writes its objective trace there."""
    c = synth.mid()
    x0 = start(c, 7)
    sched = torch.tensor(qg.qg_schedule(2 * N, 1e-2, 1e-4, 5e-2, 1e-4), device="cuda")
    tr_a = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    a = qg.Solver(c, precision=precision)
    xa = torch.tensor(x0, dtype=a.dtype, device="cuda")
    qg.qg_solve_schedule(a.h, xa, 2 * N, sched, restart=True, obj_trace=tr_a)
    b = qg.Solver(c, precision=precision)
    xb = torch.tensor(x0, dtype=b.dtype, device="cuda")
    tr_b = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    qg.qg_solve_schedule(b.h, xb, N, sched, restart=True, obj_trace=tr_b)
    blob = qg.qg_get_state(b.h)
    assert torch.equal(tr_b[:N], tr_a[:N])
    b.close()
    r = qg.Solver(c, precision=precision)
    qg.qg_set_state(r.h, blob)
    tr_r = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    qg.qg_solve_schedule(r.h, xb, N, sched, restart=False, obj_trace=tr_r)
    torch.cuda.synchronize()
    assert torch.equal(xb, xa)
    assert torch.equal(tr_r[N:], tr_a[N:])
    assert torch.count_nonzero(tr_r[:N]).item() == 0
    a.close()
    r.close()


def test_state_carries_the_screening_selection(qg):
    c = synth.mid()
    x = torch.tensor(start(c, 9), dtype=torch.float64, device="cuda")
    a = qg.Solver(c, precision=0, ctg_frac=0.3)
    Ks = int(np.ceil(0.3 * c.K))
    sel = np.sort(np.random.default_rng(4).choice(c.K, Ks, replace=False)).astype(np.int32)
    qg.qg_ctg_select(a.h, 0, sel)
    oa, ga = (t.clone() for t in a.eval_grad(x))
    r = qg.Solver(c, precision=0, ctg_frac=0.3)
    o0, g0 = (t.clone() for t in r.eval_grad(x))  # its initial selection (the first Ks outages)
    assert not torch.equal(g0, ga)
    qg.qg_set_state(r.h, qg.qg_get_state(a.h))
    orr, gr = r.eval_grad(x)
    assert torch.equal(orr, oa) and torch.equal(gr, ga)
    a.close()
    r.close()


def test_state_carries_the_rounding_state(qg):
    """Alg. 1 between rounds: the fixed pairs and the box they pinned travel in the blob."""
    c = synth.with_commitment(synth.with_block_bids(synth.tiny(), 3, 0.3, 1), 1)
    x0 = start(c, 11)
    a = qg.Solver(c, precision=0)
    xa = torch.tensor(x0, dtype=torch.float64, device="cuda")
    qg.qg_solve(a.h, xa, N, 1e-3, 0.9, 0.999)
    nf, nb = qg.qg_round_batch(a.h, xa, 0.4)
    assert 0 < nf < nb
    blob = qg.qg_get_state(a.h)
    r = qg.Solver(c, precision=0)
    plain = qg.qg_state_size(r.h)
    qg.qg_set_state(r.h, blob)
    assert qg.qg_state_size(r.h) == len(blob) > plain
    xr = xa.clone()
    qg.qg_solve(a.h, xa, N, 1e-3, 0.9, 0.999)
    qg.qg_solve(r.h, xr, N, 1e-3, 0.9, 0.999)
    torch.cuda.synchronize()
    assert torch.equal(xr, xa)
    nf2, _ = qg.qg_round_batch(r.h, xr, 0.4)  # the next round starts from the restored flags
    nf3, _ = qg.qg_round_batch(a.h, xa, 0.4)
    assert nf2 == nf3 > nf
    assert torch.equal(xr, xa)
    a.close()
    r.close()


def test_set_state_validates_the_blob(qg):
    c = synth.tiny()
    a = qg.Solver(c, precision=0)
    blob = qg.qg_get_state(a.h)
    m = qg.Solver(c, precision=1)  # another precision
    with pytest.raises(qg.QGError) as ei:
        qg.qg_set_state(m.h, blob)
    assert ei.value.code == qg.QG_ERR_INVALID_ARG
    o = qg.Solver(synth.mid(), precision=0)  # another size
    with pytest.raises(qg.QGError):
        qg.qg_set_state(o.h, blob)
    with pytest.raises(qg.QGError):
        qg.qg_set_state(a.h, blob[:-8])  # truncated
    with pytest.raises(qg.QGError):
        qg.qg_set_state(a.h, b"XXXX" + blob[4:])  # not a blob
    s = qg.Solver(c, precision=0, ctg_frac=0.5)  # screening on one side only
    with pytest.raises(qg.QGError):
        qg.qg_set_state(s.h, blob)
    qg.qg_set_state(a.h, blob)  # a valid blob still restores
    for h in (a, m, o, s):
        h.close()
