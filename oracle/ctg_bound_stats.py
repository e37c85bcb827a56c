"""How much of the contingency screen a bound test can settle (Sec. II-E; test and analysis
infrastructure: the product never imports this module).

For every period t, monitored branch m and outage k the screen's question is whether
F = f_m + L[m, k] f_k can reach the post-contingency limit: F^2 + qmax2_m - s_ctg_m^2 > 0.  A bound
test answers it for a whole piece at once: with Lmax the largest |L| of a row over a group of
outages and fc the largest |f_k| of the group over a chunk of periods, Lmax fc < sqrt(s_ctg^2 -
qmax2) - |f_m| (for every period of the chunk) rules every element of the piece out.  This module
counts, in FP64 from the oracle's own flows and line-outage block, how many elements are candidates
and which fraction of the pieces such a test clears, at the sizes the contingency kernel uses: a
warp holds 8 rows x 64 outages in 16-outage groups, a block tile 64 x 64, chunks of 8 periods.

    python -m oracle.ctg_bound_stats dayahead      # a few minutes of CPU
"""
import sys

import numpy as np

from . import qg_oracle as Q


def flows_and_block(case, x):
    """Base DC flows f (T, M), the line-outage block L (M, K) with 0 at each outage's own branch, and
    qmax2 (T, M) at x, all from the oracle."""
    v, th, p = Q.unpack(case, x)[:3]
    net = Q.dc_network(case)
    _, pbar = Q.dc_injections(case, p)
    _, f = Q.dc_base_flows(case, net, pbar)
    U, den = Q.outage_columns(case, net)
    Eh = net.E[:, net.keep]
    L = np.asarray(net.y[:, None] * (Eh @ U)) / den[None, :]
    L[case.ctg, np.arange(case.K)] = 0.0
    _, qf, _, qt = Q.ac_flows(case, v, th)
    return f, L, np.maximum(qf * qf, qt * qt)


def stats(case, x, group=16, chunk=8, warp_rows=8, tile=64, slack=1.0):
    """Candidate fraction and the fractions of (warp, chunk) pieces and (tile, chunk) items the bound
    test settles, in FP64 (the kernel's test rounds towards failing, so its own rates are at most
    these), and the number of candidates inside cleared pieces (0 for a sound test).  slack > 1 scales
    the clearance up, a deliberately loose test (for the tests that check this count can fail)."""
    f, L, q2 = flows_and_block(case, x)
    T, M, K = case.T, case.n_branch, case.K
    Mp, Kp = -(-M // tile) * tile, -(-K // tile) * tile
    A = np.zeros((Mp, Kp))
    A[:M, :K] = np.abs(L)
    lmax = A.reshape(Mp, Kp // group, group).max(axis=2)
    fk = np.zeros((T, Kp))
    fk[:, :K] = np.abs(f[:, case.ctg])
    fkmax = fk.reshape(T, Kp // group, group).max(axis=2)
    s2 = case.s_max_ctg ** 2
    clear = np.full((T, Mp), np.inf)
    with np.errstate(invalid="ignore"):
        c = np.sqrt(np.maximum(s2[None, :] - q2, 0.0)) - np.abs(f)
    c[~(c > 0)] = -1.0
    clear[:, :M] = c
    cand = tot = unsound = 0
    warp_ok = warp_n = item_fail = item_n = 0
    for t0 in range(0, T, chunk):
        t1 = min(T, t0 + chunk)
        ok = lmax * fkmax[t0:t1].max(axis=0)[None, :] < slack * clear[t0:t1].min(axis=0)[:, None]
        okw = ok.reshape(Mp // warp_rows, warp_rows, Kp // tile, tile // group).all(axis=(1, 3))
        cleared = np.repeat(np.repeat(okw, warp_rows, axis=0), tile, axis=1)[:M, :K]  # per element
        for t in range(t0, t1):
            F = f[t][:, None] + L * f[t][case.ctg][None, :]
            y = F * F + (q2[t] - s2)[:, None]
            y[case.ctg, np.arange(K)] = -1.0          # the outaged branch is not monitored
            cand += int((y > 0).sum())
            unsound += int(((y > 0) & cleared).sum())
            tot += M * K - K
        warp_ok += int(okw.sum())
        warp_n += okw.size
        fails = ~okw.reshape(Mp // tile, tile // warp_rows, Kp // tile).all(axis=1)
        item_fail += int(fails.sum())
        item_n += fails.size
    return {"candidate_fraction": cand / tot, "candidates": cand, "candidates_in_cleared_pieces": unsound,
            "warp_chunks_cleared": warp_ok / warp_n, "tile_chunks_with_a_failing_warp": item_fail / item_n}


def main(argv):
    import synth
    from .copperplate import lambda_dispatch
    name = argv[1] if len(argv) > 1 else "dayahead"
    case = getattr(synth, name)()
    print(name, stats(case, case.flat_start(lambda_dispatch(case))))  # economic dispatch, flat voltage


if __name__ == "__main__":
    main(sys.argv)
