"""Writes the thermal ratings and copper-plate starts of the named synthetic cases
(run by hand; output is committed).

TEST INFRASTRUCTURE (see qg_oracle.py).  For each case the generator draws every
input except the ratings; this script dispatches generation in merit order
(oracle.copperplate.lambda_dispatch), computes the base-case DC branch flows with
the oracle's own solve (Sec. II-E, Eq. Yb_solve/p_flow) and sets
    s_max_j = s_max_ctg_j = max(RATING_FLOOR, RATING_MARGIN * max_t |f_jt|),
stored as float32 in synth/ratings/<case name>.npy.  The generator reads them back.

For the cases the tests and the benchmark start from (tiny14, mid150, rt617) it
also stores the copper-plate dispatch of Sec. III-A (oracle.copperplate, exact
tangent-cut QP) and its bound in synth/ratings/<case name>_lp.npz: the start
x0 = (flat voltage, zero angles and q, copper-plate p and r) and the reference
value of the "within 1% of the LP bound" metric.

    python -m oracle.make_ratings            # every named case
"""
from __future__ import annotations

import os
import sys

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .copperplate import copper_plate, lambda_dispatch

RATING_MARGIN = 2.0
RATING_FLOOR = 0.5
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "synth", "ratings")


def dc_flows_sparse(case, p):
    """Base-case DC flows with the uniform slack, via a sparse factorisation (large cases)."""
    n, M = case.n_bus, case.n_branch
    y = case.br_x / (case.br_r ** 2 + case.br_x ** 2)
    E = sp.csr_matrix((np.r_[np.ones(M), -np.ones(M)],
                       (np.r_[np.arange(M), np.arange(M)], np.r_[case.br_from, case.br_to])), shape=(M, n))
    keep = np.array([i for i in range(n) if i != case.ref_bus])
    Eh = E[:, keep]
    Y = (Eh.T @ sp.diags(y) @ Eh).tocsc()
    lu = spla.splu(Y)
    inj = -case.load_p.copy()
    np.add.at(inj.T, case.gen_bus, p.T)
    pbar = inj - inj.mean(axis=1, keepdims=True)
    th = np.zeros_like(pbar)
    th[:, keep] = lu.solve(pbar[:, keep].T).T
    return (E @ th.T).T * y[None, :]


def ratings_for(case):
    p = lambda_dispatch(case)
    f = dc_flows_sparse(case, p)
    return np.maximum(RATING_FLOOR, RATING_MARGIN * np.abs(f).max(axis=0)).astype(np.float32)


def main(argv):
    sys.path.insert(0, os.path.dirname(HERE))
    import synth
    os.makedirs(OUT, exist_ok=True)
    cases = [synth.tiny(), synth.mid(), synth.rt617()] + synth.batch()
    if "--no-large" not in argv:
        cases.append(synth.dayahead())
    for c in cases:
        r = ratings_for(c)
        np.save(os.path.join(OUT, c.name + ".npy"), r)
        print(c.name, c.n_branch, float(r.min()), float(r.max()))
    for mk in (synth.tiny, synth.mid, synth.rt617):
        c = mk()
        bound, p, rr = copper_plate(c)
        np.savez(os.path.join(OUT, c.name + "_lp.npz"), p=p, r=rr, bound=np.array(bound))
        print(c.name, "copper-plate bound", bound)


if __name__ == "__main__":
    main(sys.argv[1:])
