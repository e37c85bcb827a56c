"""The running-list policy of Alg. 2 (screening.ContingencyScreen) on the host: scores of the last
evaluation update the list, unscored outages rank first, the next subset is the top fraction plus a
seeded random draw from the rest, always Ks distinct outages.  The device call is replaced by a
recorder (no GPU)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def screening():
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import screening as mod
    return mod


def test_running_list_policy(screening, monkeypatch):
    calls = []
    monkeypatch.setattr(screening.qg, "qg_ctg_select", lambda h, inst, sel: calls.append(np.array(sel)))
    T, K, Ks = 3, 20, 8
    scr = screening.ContingencyScreen(h=0, T=T, K=K, Ks=Ks, inst=0, top_frac=0.5, seed=7)
    assert np.array_equal(scr.sel, np.arange(Ks))
    rng = np.random.default_rng(0)
    z = rng.uniform(0, 1, size=(T, Ks))
    scr.update(z.ravel())
    np.testing.assert_array_equal(scr.score[:Ks], z.max(axis=0))       # max over the periods
    assert np.all(np.isinf(scr.score[Ks:]))                            # unscored: +inf, rank first
    sel = scr.select()
    assert len(sel) == Ks == len(set(sel.tolist())) and np.all(np.diff(sel) > 0)
    assert set(range(Ks, Ks + 4)) <= set(sel.tolist())                  # the 4 top ranks: unscored ones
    assert np.array_equal(calls[-1], sel)
    # scored everywhere: the top half are the largest scores, the rest a seeded draw
    scr.score = np.arange(K, dtype=float)
    sel2 = scr.select()
    assert set(range(K - 4, K)) <= set(sel2.tolist())
    scr2 = screening.ContingencyScreen(h=0, T=T, K=K, Ks=Ks, inst=0, top_frac=0.5, seed=7)
    scr2.score = np.arange(K, dtype=float)
    scr2.rng = np.random.default_rng(7)
    scr.rng = np.random.default_rng(7)
    assert np.array_equal(scr.select(), scr2.select())                 # deterministic for a seed
