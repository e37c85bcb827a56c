"""Batch rounding (Alg. 1) with the per-pair projection stand-in through the C ABI, against the
oracle of one round (oracle/rounding.py): the same pairs fixed, the same projected values, the box
holding them through later Adam steps, and the full loop ending with every binary fixed."""
import numpy as np
import pytest

import oracle
import synth
from oracle import rounding as R

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


def case(seed=1, base=synth.tiny):
    return synth.with_commitment(synth.with_block_bids(base(), 3, 0.3, seed), seed=seed)


def start(c, seed):
    """Inside the box; p spread over [0, pmax] (the box with on-status), u uniform: both choices occur."""
    x = synth.random_point(c, seed)
    o = c.offsets()
    rng = np.random.default_rng(seed)
    x[o[2]:o[3]] = (rng.uniform(size=(c.T, c.n_gen)) * c.pmax).ravel()
    lo, hi = oracle.box(c)
    return np.clip(x, lo, hi)


def apply_oracle_round(c, x, fixed, frac):
    u, p, q, r, d = R.project_binaries(c, x)
    d = np.where(fixed, np.inf, d)
    pick = R.select(d, fixed, frac)
    xn = x.copy()
    o = c.offsets()
    ou = c.offset_u()
    TG = c.T * c.n_gen
    for name, arr, off in (("p", p, o[2]), ("q", q, o[3]), ("r", r, o[4]), ("u", u, ou)):
        xn[off + pick] = arr.ravel()[pick]
    fixed = fixed.copy().ravel()
    fixed[pick] = True
    return xn, fixed.reshape(c.T, c.n_gen), pick, TG


def test_two_rounds_match_the_oracle(qg):
    c = case()
    x0 = start(c, 3)
    s = qg.Solver(c, precision=0)
    x = torch.tensor(x0, dtype=torch.float64, device="cuda")
    fixed = np.zeros((c.T, c.n_gen), bool)
    xr = x0
    for rnd, frac in enumerate((0.3, 0.5)):
        nf, nb = qg.qg_round_batch(s.h, x, frac)
        xr, fixed, pick, TG = apply_oracle_round(c, xr, fixed, frac)
        assert nb == TG and nf == fixed.sum(), (rnd, nf, fixed.sum())
        np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=0, atol=1e-14)
    u = oracle.unpack_u(c, xr)
    assert 0 < (u[fixed] == 0).sum() < fixed.sum()  # both choices among the fixed pairs
    s.close()


def test_the_box_holds_fixed_pairs_through_adam(qg):
    c = case(2)
    x0 = start(c, 5)
    s = qg.Solver(c, precision=0)
    x = torch.tensor(x0, dtype=torch.float64, device="cuda")
    qg.qg_round_batch(s.h, x, 0.5)
    xf = x.cpu().numpy().copy()
    _, _, _, _, d = R.project_binaries(c, x0)
    pick = R.select(d, np.zeros_like(d, bool), 0.5)
    qg.qg_solve(s.h, x, 30, 1e-2, 0.9, 0.999)
    xs = x.cpu().numpy()
    o, ou = c.offsets(), c.offset_u()
    np.testing.assert_array_equal(xs[ou + pick], xf[ou + pick])              # u pinned
    off = pick[xf[ou + pick] == 0]
    for k in (o[2], o[3], o[4]):
        np.testing.assert_array_equal(xs[k + off], 0.0)                      # off: p = q = r = 0
    on = pick[xf[ou + pick] == 1]
    assert np.all(xs[o[2] + on] >= np.tile(c.pmin, c.T)[on] - 1e-15)         # on: p >= pmin now
    free = np.setdiff1d(np.arange(c.T * c.n_gen), pick)
    assert np.max(np.abs(xs[ou + free] - xf[ou + free])) > 1e-3             # unfixed u still move
    qg.qg_round_reset(s.h)
    qg.qg_solve(s.h, x, 30, 1e-2, 0.9, 0.999)
    assert np.max(np.abs(x.cpu().numpy()[ou + pick] - xf[ou + pick])) > 1e-3  # reset frees them
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_rounding_loop_fixes_every_binary(qg, precision):
    from paper_2310_06650_gb300.rounding import batch_round
    c = case(4, base=synth.mid)
    x0 = start(c, 8)
    s = qg.Solver(c, precision=precision)
    x = torch.tensor(x0, dtype=s.dtype, device="cuda")
    rounds = batch_round(s, x, frac=0.34, iters=50, lr=1e-3, final_iters=20)
    assert rounds[-1][0] == rounds[-1][1] == c.T * c.n_gen and len(rounds) <= 20
    assert all(a[0] < b[0] for a, b in zip(rounds, rounds[1:]))  # every round fixes more
    xs = x.double().cpu().numpy()
    u = oracle.unpack_u(c, xs)
    assert set(np.unique(u)) <= {0.0, 1.0}
    _, _, p, q, r = oracle.unpack(c, xs)
    assert np.all(p[u == 0] == 0) and np.all(q[u == 0] == 0) and np.all(r[u == 0] == 0)
    pm = np.broadcast_to(c.pmin, p.shape)
    assert np.all(p[u == 1] >= pm[u == 1] - 1e-6)
    res = oracle.evaluate(c, xs)
    assert np.isfinite(res.obj)
    s.close()


def test_rounding_skips_instances_without_on_status(qg):
    c = synth.tiny()
    s = qg.Solver([c, case()], precision=0)
    x = torch.tensor(np.concatenate([c.flat_start(), start(case(), 1)]), dtype=torch.float64, device="cuda")
    nf, nb = qg.qg_round_batch(s.h, x, 1.0)
    assert nb == case().T * case().n_gen and nf == nb
    np.testing.assert_array_equal(x.cpu().numpy()[:c.n_x], c.flat_start())
    s.close()
    s = qg.Solver(c, precision=0)
    x = torch.tensor(c.flat_start(), dtype=torch.float64, device="cuda")
    assert qg.qg_round_batch(s.h, x, 0.5) == (0, 0)
    s.close()
