"""Contingency screening of Alg. 2 on top of a screening handle (qg_options.ctg_frac in (0, 1)).

The library evaluates a fixed-size subset of every instance's outages (qg_ctg_select) and reports
the scores of the evaluated ones (qg_ctg_scores).  This module keeps Alg. 2's running list: each
outage's latest score (the largest over the periods of its last evaluation); unscored outages rank
first.  The next subset is the top `top_frac` of the list plus a seeded random draw from the rest
(the stochastic selection), one subset for all periods of the instance.
"""
from __future__ import annotations

import numpy as np

from . import qg


class ContingencyScreen:
    def __init__(self, h: int, T: int, K: int, Ks: int, inst: int = 0, top_frac: float = 0.5, seed: int = 0):
        self.h, self.T, self.K, self.Ks, self.inst = h, T, K, Ks, inst
        self.n_top = min(Ks, int(round(top_frac * Ks)))
        self.score = np.full(K, np.inf)
        self.rng = np.random.default_rng(seed)
        self.sel = np.arange(Ks, dtype=np.int32)

    def update(self, z: np.ndarray) -> None:
        """z: this instance's scores of the last evaluation, T x Ks in the order of the selection."""
        self.score[self.sel] = np.asarray(z).reshape(self.T, self.Ks).max(axis=0)

    def select(self) -> np.ndarray:
        order = np.argsort(-self.score, kind="stable")
        top = order[:self.n_top]
        rest = order[self.n_top:]
        extra = self.rng.choice(rest, size=self.Ks - self.n_top, replace=False) if self.Ks > self.n_top else []
        self.sel = np.sort(np.concatenate([top, extra]).astype(np.int32))
        qg.qg_ctg_select(self.h, self.inst, self.sel)
        return self.sel


def screened_solve(solver, x, iters: int, every: int, lr: float = 1e-3, top_frac: float = 0.5, seed: int = 0,
                   table=None):
    """Adam on a single-instance screening handle: `every` iterations per subset, then the subset is
    re-drawn from the updated list.  With a schedule table the run follows it (qg_solve_schedule)."""
    c = solver.cases[0]
    Ks = max(1, int(np.ceil(solver.ctg_frac * c.K)))
    scr = ContingencyScreen(solver.h, c.T, c.K, Ks, 0, top_frac, seed)
    done = 0
    while done < iters:
        n = min(every, iters - done)
        if table is not None:
            qg.qg_solve_schedule(solver.h, x, n, table, done == 0, 0.9, 0.999)
        else:
            qg.qg_solve(solver.h, x, n, lr, 0.9, 0.999)
        done += n
        scr.update(qg.qg_ctg_scores(solver.h, c.T * Ks))
        scr.select()
    return scr
