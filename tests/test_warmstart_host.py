"""Host helpers of the warm-start pipeline against the oracle: the merit-order start and its bound
(the library's own copper-plate dispatch without reserve and ramp terms) against the oracle's KKT
dispatch and its exact copper-plate bound, and the time-to-target reading of a trace."""
import numpy as np
import pytest

import synth
from oracle.copperplate import copper_plate, lambda_dispatch


@pytest.fixture(scope="module")
def warmstart():
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import warmstart as mod
    return mod


@pytest.mark.parametrize("mk", [synth.tiny, synth.mid])
def test_merit_order_dispatch_matches_the_oracle_kkt_dispatch(warmstart, mk):
    c = mk()
    p = warmstart.merit_order_dispatch(c)
    np.testing.assert_allclose(p, lambda_dispatch(c), rtol=0, atol=1e-8 * c.pmax.max())
    np.testing.assert_allclose(p.sum(axis=1), c.load_p.sum(axis=1), rtol=1e-10)


def test_merit_order_bound_is_below_the_copper_plate_bound(warmstart):
    """Dropping the reserve terms can only lower the copper-plate optimum."""
    c = synth.tiny()
    bound, _, _ = copper_plate(c)
    assert warmstart.merit_order_bound(c) <= bound * (1 + 1e-9)


def test_time_to_target(warmstart):
    t = np.array([1.0, 2.0, 3.0, 4.0])
    o = np.array([9.0, 5.0, 6.0, 2.0])
    assert warmstart.time_to(t, o, 5.5) == 2.0
    assert warmstart.time_to(t, o, 2.0) == 4.0
    assert warmstart.time_to(t, o, 1.0) == float("inf")
