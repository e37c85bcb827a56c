"""Pins of the batch-rounding oracle (Alg. 1 with the per-pair projection stand-in).

The limit projection is checked by the variational inequality that characterizes a Euclidean
projection onto a convex polygon, (x0 - y) . (z - y) <= 0 at every vertex z, found by intersecting
the constraint lines; the on/off choice against a dense grid search; the selection against a
sort of (distance, index) pairs."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from oracle import rounding as R


def _vertices(pmin, pmax, rcap):
    """Vertices of {pmin <= p <= pmax, 0 <= r <= rcap, p + r <= pmax}: feasible pairwise
    intersections of its constraint lines (a p + b r = c)."""
    lines = [(1, 0, pmin), (1, 0, pmax), (0, 1, 0.0), (0, 1, rcap), (1, 1, pmax)]
    out = []
    for (a1, b1, c1), (a2, b2, c2) in itertools.combinations(lines, 2):
        det = a1 * b2 - a2 * b1
        if abs(det) < 1e-15:
            continue
        p = (c1 * b2 - c2 * b1) / det
        r = (a1 * c2 - a2 * c1) / det
        if pmin - 1e-12 <= p <= pmax + 1e-12 and -1e-12 <= r <= rcap + 1e-12 and p + r <= pmax + 1e-12:
            out.append((p, r))
    return out


@pytest.mark.parametrize("seed", range(5))
def test_limit_projection_satisfies_the_variational_inequality(seed):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        pmax = rng.uniform(0.5, 3.0)
        pmin = rng.uniform(0.0, 0.6) * pmax
        rcap = pmax if rng.uniform() < 0.8 else 0.0
        p0, r0 = rng.uniform(-1, 4), rng.uniform(-1, 4)
        p, r = R.project_on(np.array([p0]), np.array([r0]), pmin, pmax, rcap)
        p, r = float(p[0]), float(r[0])
        assert pmin - 1e-12 <= p <= pmax + 1e-12 and -1e-12 <= r <= rcap + 1e-12 and p + r <= pmax + 1e-12
        for zp, zr in _vertices(pmin, pmax, rcap):
            assert (p0 - p) * (zp - p) + (r0 - r) * (zr - r) <= 1e-10


def _case():
    return synth.with_commitment(synth.with_block_bids(synth.tiny(), 3, 0.3, 1), seed=1)


def test_on_off_choice_matches_a_grid_search():
    c = _case()
    x = synth.random_point(c, 4)
    # push some points outside the limits so that both choices occur
    o = c.offsets()
    x[o[2]:o[3]] *= np.random.default_rng(1).uniform(-0.3, 1.4, size=c.T * c.n_gen)
    u, p, q, r, d = R.project_binaries(c, x)
    _, _, p0, q0, r0 = oracle.unpack(c, x)
    u0 = oracle.unpack_u(c, x)
    cons = oracle.device_sign(c) < 0
    assert 0 < u.sum() < u.size
    for t in range(c.T):
        for g in range(c.n_gen):
            rcap = 0.0 if cons[g] else c.pmax[g]
            pp, rr = np.meshgrid(np.linspace(c.pmin[g], c.pmax[g], 201), np.linspace(0.0, rcap, 201))
            ok = pp + rr <= c.pmax[g] + 1e-12
            qq = np.clip(q0[t, g], c.qmin[g], c.qmax[g])
            grid1 = ((pp - p0[t, g]) ** 2 + (rr - r0[t, g]) ** 2)[ok].min() + (qq - q0[t, g]) ** 2 + (u0[t, g] - 1) ** 2
            d0 = p0[t, g] ** 2 + q0[t, g] ** 2 + r0[t, g] ** 2 + u0[t, g] ** 2
            assert d[t, g] <= min(grid1, d0) + 1e-12          # nothing on the grid beats the closed form
            if u[t, g] == 0:
                assert p[t, g] == q[t, g] == r[t, g] == 0.0 and d[t, g] == d0
            assert d[t, g] >= min(grid1, d0) - 2e-3 * max(1.0, c.pmax[g]) ** 2  # and the grid gets close


def test_selection_is_smallest_distance_then_index():
    rng = np.random.default_rng(3)
    dist = rng.integers(0, 5, size=(6, 7)).astype(float)  # many ties
    fixed = rng.uniform(size=(6, 7)) < 0.3
    for frac in (0.1, 0.25, 0.5, 1.0):
        got = R.select(dist, fixed, frac)
        free = [i for i in range(dist.size) if not fixed.ravel()[i]]
        want = sorted(sorted(free, key=lambda i: (dist.ravel()[i], i))[:int(np.ceil(frac * len(free)))])
        assert list(got) == want


def test_planted_box_only_projection_is_caught(monkeypatch):
    monkeypatch.setattr(R, "project_on", lambda p0, r0, pmin, pmax, rcap: (np.clip(p0, pmin, pmax),
                                                                           np.clip(r0, 0.0, rcap)))
    with pytest.raises(AssertionError):
        test_limit_projection_satisfies_the_variational_inequality(0)
