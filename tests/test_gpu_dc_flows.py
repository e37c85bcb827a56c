"""The base DC flows f_t (Eq. p_flow with the uniform slack of Sec. II-E) in isolation, through
qg_dc_flows, against the FP64 oracle, on the dense DC mode of both paths.

The contingency screen and every post-contingency flow start from these values, and on the mixed
path they are the one place where cancellation is large: a flow is a sum of PTDF entries times
injections of both signs, and on rt617 the sum of the terms' magnitudes is up to 2 x 10^6 times the
flow it leaves.  The mixed path forms it from double-FP32 operands (PTDF columns, load products, row sums
and total loads made in FP64 on the host, the dispatch p from the FP32 x) and rounds the result once
to FP32.  The bound checked, element by element, is half an FP32 ulp of f plus 2^-36 of the sum of
the products' magnitudes S = sum_i |PTDF_mi| (|p_i| + |load_i|) + |mu_t| sum_i |PTDF_mi|.  That is a
double-FP32 accumulation error with a 2^8 margin; the error of FP32 accumulation is a median
750-1,000 times 2^-36 S on these grids.  With phase shifters the mixed path also rounds b phi once to FP32,
and that term, 2^-24 of |PSDF| |b phi| + |b phi|, is added to the bound.  The FP64 path computes the
flows in FP64 and rounds them once.

The test also checks its own teeth: the same flows accumulated in plain FP32 (PTDF and injections
rounded to FP32, FP32 products and sums) exceed the bound on many elements of both grids."""
import functools

import numpy as np
import pytest

import oracle
import synth
from oracle import qg_oracle

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


@functools.lru_cache(maxsize=None)
def case_named(name):
    return {"mid": synth.mid, "rt617": synth.rt617,
            "mid_xf": lambda: synth.with_transformers(synth.mid(), 0.15, 5)}[name]()


def point(case, seed=11):
    lo, hi = oracle.box(case)
    return np.clip(synth.random_point(case, seed), lo, hi)


def reference(case, x):
    """Oracle flows f (T, M) and the magnitudes of the terms the device sums: S (T, M) and, with phase
    shifters, the b phi part P (T, M).  Also the plain FP32 flows (the teeth)."""
    parts = oracle.unpack(case, x)
    p = parts[2]
    net = oracle.dc_network(case, sparse=False)
    inj, pbar = oracle.dc_injections(case, p)
    bflow = None
    if len(parts) == 7:
        bflow = qg_oracle.phase_shift_flows(case, net, qg_oracle.branch_tau_phi(case, parts[5], parts[6])[1])
    _, f = oracle.dc_base_flows(case, net, pbar, bflow)
    n = case.n_bus
    Z = np.zeros((n, n))
    Z[np.ix_(net.keep, net.keep)] = net.Yinv
    ptdf = net.y[:, None] * (net.E @ Z)                       # (M, n): flow per unit injection at each bus
    gen_abs = np.zeros((case.T, n))
    np.add.at(gen_abs.T, case.gen_bus, np.abs(p).T)
    load_abs = np.abs(case.load_p)
    mu_abs = (gen_abs.sum(axis=1) + load_abs.sum(axis=1)) / n
    aptdf = np.abs(ptdf)
    S = (gen_abs + load_abs) @ aptdf.T + mu_abs[:, None] * aptdf.sum(axis=1)[None, :]
    P = np.zeros_like(f)
    if bflow is not None:
        P = np.abs(bflow) @ np.abs(net.E @ ptdf.T) + np.abs(bflow)
    # plain FP32: the same sum with every operand rounded to FP32 and FP32 arithmetic throughout
    inj32 = -case.load_p.astype(np.float32)
    np.add.at(inj32.T, case.gen_bus, (oracle.device_sign(case) * p).astype(np.float32).T)
    pbar32 = inj32 - inj32.mean(axis=1, dtype=np.float32, keepdims=True)
    naive = pbar32 @ ptdf.astype(np.float32).T
    return f, S, P, naive


def device_flows(qg, case, x, precision):
    s = qg.Solver(case, precision=precision, dc_solver=1)
    try:
        xt = torch.tensor(x, dtype=s.dtype, device="cuda")
        s.eval_grad(xt)
        torch.cuda.synchronize()
        out = qg.qg_dc_flows(s.h, case.T * case.n_branch)
    finally:
        s.close()
    return out.astype(np.float64).reshape(case.T, case.n_branch)


def bound(f, S, P, mixed):
    b = 2.0 ** -24 * np.abs(f) * (1 + 2.0 ** -20) + 2.0 ** -36 * S
    return b + 2.0 ** -24 * P if mixed else b


@pytest.mark.parametrize("name", ["mid", "rt617", "mid_xf"])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_dc_flows_within_one_fp32_rounding_of_fp64(qg, name, precision):
    c = case_named(name)
    x = point(c)
    mixed = precision == "mixed"
    if mixed:
        x = np.asarray(x, dtype=np.float32).astype(np.float64)   # the mixed path holds x in FP32
    f, S, P, naive = reference(c, x)
    got = device_flows(qg, c, x, qg.QG_MIXED if mixed else qg.QG_FP64)
    tol = bound(f, S, P, mixed)
    err = np.abs(got - f)
    worst = np.unravel_index(np.argmax(err / tol), err.shape)
    assert np.all(err <= tol), (name, precision, worst, got[worst], f[worst], tol[worst])
    # the test's teeth: plain FP32 accumulation of the same flows misses the bound on many elements
    if name != "mid_xf":
        miss = np.abs(naive - f) > bound(f, S, P, True)
        assert miss.mean() > 0.05, (name, miss.mean())


def test_dc_flows_batched_layout(qg):
    """A batch of two instances: the flows come back instance-major, each instance [T][M]."""
    cs = [case_named("mid"), synth.tiny()]
    xs = [np.asarray(point(c, 5 + i), dtype=np.float32).astype(np.float64) for i, c in enumerate(cs)]
    s = qg.Solver(cs, precision=qg.QG_MIXED, dc_solver=1)
    try:
        xt = torch.tensor(np.concatenate(xs), dtype=s.dtype, device="cuda")
        s.eval_grad(xt)
        torch.cuda.synchronize()
        out = qg.qg_dc_flows(s.h, sum(c.T * c.n_branch for c in cs)).astype(np.float64)
    finally:
        s.close()
    o = 0
    for c, x in zip(cs, xs):
        f, S, P, _ = reference(c, x)
        got = out[o:o + c.T * c.n_branch].reshape(c.T, c.n_branch)
        o += c.T * c.n_branch
        assert np.all(np.abs(got - f) <= bound(f, S, P, True)), c.n_bus
