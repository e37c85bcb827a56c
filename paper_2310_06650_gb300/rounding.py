"""Batch rounding of the relaxed on-status variables (Alg. 1) on a handle whose instances have them.

Each round solves the continuous problem with the already fixed binaries held by the clip box
(graph-replayed Adam, qg_solve or a scheduled qg_solve_schedule), then projects every unfixed binary
with the library's per-pair projection stand-in and fixes the fraction `frac` of them that moved
least (qg_round_batch), until every binary is fixed; a last solve polishes the continuous variables.
"""
from __future__ import annotations

from . import qg


def batch_round(solver, x, frac: float = 0.25, iters: int = 200, lr: float = 1e-3, beta1: float = 0.9,
                beta2: float = 0.999, final_iters: int = 0, max_rounds: int = 1000):
    """Alg. 1 on `solver` (a qg.Solver) from the device point x (updated in place).  Returns the
    per-round (fixed, total) pair counts."""
    rounds = []
    for _ in range(max_rounds):
        qg.qg_solve(solver.h, x, iters, lr, beta1, beta2)
        nf, nb = qg.qg_round_batch(solver.h, x, frac)
        rounds.append((nf, nb))
        if nf >= nb:
            break
    if final_iters:
        qg.qg_solve(solver.h, x, final_iters, lr, beta1, beta2)
    return rounds
