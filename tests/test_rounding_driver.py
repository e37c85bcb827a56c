"""The Alg. 1 loop of rounding.batch_round on the host: a solve, then one rounding round, until every
binary is fixed, then the optional polishing solve; the device calls are replaced by recorders."""
import math

import pytest


@pytest.fixture(scope="module")
def rounding():
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import rounding as mod
    return mod


class _Solver:
    h = 0


def test_loop_alternates_solves_and_rounds_until_all_fixed(rounding, monkeypatch):
    log = []
    state = {"fixed": 0}
    n_bin = 37

    def solve(h, x, iters, lr, b1, b2):
        log.append(("solve", iters))

    def round_batch(h, x, frac):
        state["fixed"] += math.ceil(frac * (n_bin - state["fixed"]))
        log.append(("round", frac))
        return state["fixed"], n_bin

    monkeypatch.setattr(rounding.qg, "qg_solve", solve)
    monkeypatch.setattr(rounding.qg, "qg_round_batch", round_batch)
    rounds = rounding.batch_round(_Solver(), None, frac=0.5, iters=10, final_iters=5)
    assert rounds[-1] == (n_bin, n_bin) and all(a[0] < b[0] for a, b in zip(rounds, rounds[1:]))
    kinds = [k for k, _ in log]
    assert kinds == ["solve", "round"] * len(rounds) + ["solve"]
    assert log[-1] == ("solve", 5)
