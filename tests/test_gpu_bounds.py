"""The index-checked build (QG_CHECK_BOUNDS; `python -m paper_2310_06650_gb300.build --check-bounds`):
every access d.<array>[i] of the stage kernels is checked against the address ranges of the
library's device arrays and the caller's arrays a handle holds; a miss would be recorded and
redirected to a dummy word.  Small cases of every kernel family run on that build in a child
process (the library is chosen by QG_LIBRARY at import) and are compared with the oracle; no checked
access may miss."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, ROOT)
import numpy as np, torch
import oracle, synth
from paper_2310_06650_gb300 import qg

def point(c, seed):
    return np.clip(synth.random_point(c, seed), *oracle.box(c))

def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))

res = {}
def run(name, cases, prec, seed, **kw):
    cases = cases if isinstance(cases, list) else [cases]
    xs = [point(c, seed + i) for i, c in enumerate(cases)]
    s = qg.Solver(cases, precision=prec, **kw)
    x = torch.tensor(np.concatenate(xs), dtype=s.dtype, device="cuda")
    obj, g = (t.clone() for t in s.eval_grad(x))
    torch.cuda.synchronize()
    refs = [oracle.evaluate(c, xx) for c, xx in zip(cases, xs)]
    tol = 1e-9 if prec == qg.QG_FP64 else 1e-4
    ro = max(rel(obj[b].item(), r.obj) for b, r in enumerate(refs))
    rg = rel(g.double().cpu().numpy(), np.concatenate([r.grad for r in refs]))
    trace = torch.zeros(9 * len(cases), dtype=torch.float64, device="cuda")
    qg.qg_solve(s.h, x, 9, 1e-3, 0.9, 0.999, trace)       # graph-replayed iterations with a trace
    qg.qg_solve(s.h, x, 9, 1e-3, 0.9, 0.999)              # and without (the shared closing kernel)
    torch.cuda.synchronize()
    s.close()
    res[name] = (ro, rg, tol)

for prec in (qg.QG_FP64, qg.QG_MIXED):
    run(f"tiny {prec}", synth.tiny(), prec, 1)
    run(f"mid {prec}", synth.mid(), prec, 2)
    run(f"mid sparse {prec}", synth.mid(), prec, 3, dc_solver=qg.QG_DC_SPARSE)
    run(f"mid screened {prec}", synth.mid(), prec, 4, ctg_frac=1.0 - 1e-9)
    dev = synth.with_commitment(synth.with_block_bids(synth.with_transformers(synth.tiny(), 0.3, 4), 3, 0.3, 1), 1)
    run(f"devices {prec}", dev, prec, 5)
    run(f"ragged batch {prec}", [synth.tiny(), synth.mid(), synth.tiny()], prec, 6)
# a scheduled solve (the schedule table is a caller's array the kernels read)
c = synth.mid()
s = qg.Solver(c, precision=qg.QG_MIXED)
x = torch.tensor(point(c, 7), dtype=torch.float32, device="cuda")
sched = torch.tensor(qg.qg_schedule(12, 1e-2, 1e-4, 5e-2, 1e-4), device="cuda")
qg.qg_solve_schedule(s.h, x, 12, sched, restart=True)
torch.cuda.synchronize()
s.close()
print(json.dumps({"cases": res, "report": qg.qg_bounds_report()}))
"""


def test_checked_build_sees_no_bad_index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_06650_gb300.build import build
    lib = build(check_bounds=True)
    env = dict(os.environ, QG_LIBRARY=lib)
    out = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                         text=True, timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["report"] is None, f"a checked access missed: line {res['report'][0]} of qg_kernels.cu"
    for name, (ro, rg, tol) in res["cases"].items():
        assert ro <= tol and rg <= tol, (name, ro, rg)
