"""Host-side sizing of the on-demand contingency path: the clearance minima of k_ctg_margin live in T
rows of n_mt 64 floats per instance, indexed by chunk q = tci NCH + ch with NCH = ceil(ctg_tb / 8).
For every horizon and every period split the planner can produce (ctg_tb = ceil(T / ntc), ctg_ntc =
ceil(T / ctg_tb)), the chunks must fit in those T rows and cover each period exactly once."""


def ceil_div(a, b):
    return -(-a // b)


def test_chunks_fit_and_cover_every_period_once():
    for T in range(1, 97):
        for ntc in range(1, T + 1):
            tb = ceil_div(T, ntc)
            n_tc = ceil_div(T, tb)
            nch = ceil_div(tb, 8)
            assert n_tc * nch <= T, (T, ntc, tb, n_tc, nch)
            seen = [0] * T
            for tci in range(n_tc):
                t0 = tci * tb
                TB = min(tb, T - t0)
                for ch in range(nch):
                    ta, tz = t0 + ch * 8, t0 + min(TB, ch * 8 + 8)
                    assert tci * nch + ch < T
                    for t in range(ta, tz):
                        seen[t] += 1
            assert seen == [1] * T, (T, ntc)
