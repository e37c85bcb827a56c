"""The oracle against its committed regression record (tests/golden/oracle_regression.json, written
by tests/golden/make_golden.py from the oracle alone).  Not a pin (those are the closed forms,
re-solves, LPs and finite differences of the other oracle tests): it flags any change of the oracle's
arithmetic, which then has to be justified by the paper and the record rewritten."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_matches_its_regression_record():
    with open(os.path.join(HERE, "golden", "oracle_regression.json")) as f:
        want = json.load(f)
    got = make_golden.records()
    assert sorted(got) == sorted(want)
    for key, w in want.items():
        g = got[key]
        assert abs(g["obj"] - w["obj"]) <= 1e-12 * abs(w["obj"]), key
        for term, v in w["terms"].items():
            assert abs(g["terms"][term] - v) <= 1e-12 * max(abs(v), 1e-12 * abs(w["obj"])), (key, term)
        assert g["grad_idx"] == w["grad_idx"]
        np.testing.assert_allclose(g["grad"], w["grad"], rtol=1e-11, atol=1e-12 * np.abs(w["grad"]).max())
