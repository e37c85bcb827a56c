"""The bound test of the contingency screen, in FP64 on the oracle's own values (oracle/ctg_bound_stats.py):
sound (no candidate inside a cleared piece) on rt617 at the economic-dispatch start, and the count
that shows it can fail: a clearance taken twice too large clears pieces that hold candidates."""
import synth
from oracle.copperplate import lambda_dispatch
from oracle.ctg_bound_stats import stats


def _x(case):
    return case.flat_start(lambda_dispatch(case))


def test_bound_is_sound_on_rt617():
    c = synth.rt617()
    r = stats(c, _x(c))
    assert r["candidates"] > 0 and r["candidates_in_cleared_pieces"] == 0, r
    assert 0.05 < r["warp_chunks_cleared"] < 0.5, r
    assert 0.0 <= r["tile_chunks_with_a_failing_warp"] <= 1.0


def test_a_loose_bound_is_caught():
    c = synth.rt617()
    r = stats(c, _x(c), slack=2.0)
    assert r["candidates_in_cleared_pieces"] > 0, r
