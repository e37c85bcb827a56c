"""Writes tests/golden/oracle_regression.json: the oracle's objective terms and a few gradient entries
at seeded points of the tiny case and of its device-model and transformer variants.

A regression record of the oracle (calls only oracle/ and synth/), not a pin: the pins of the oracle
are the closed forms, brute-force re-solves, LPs and finite differences in tests/test_oracle_*.py.
A change of the oracle's arithmetic that moves these numbers must name, in its commit message, the
passage of the paper that justifies it, and rewrite this file with this script.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = {
    "tiny": lambda: synth.tiny(),
    "tiny_xf": lambda: synth.with_transformers(synth.tiny(), 0.3, 4),
    "tiny_devices": lambda: synth.with_commitment(synth.with_block_bids(synth.tiny(), 3, 0.3, 1), seed=1),
}
SEEDS = (1, 2)
PROBE = 12  # gradient entries recorded per point (evenly spaced)


def records():
    out = {}
    for name, mk in CASES.items():
        c = mk()
        for seed in SEEDS:
            x = synth.random_point(c, seed)
            r = oracle.evaluate(c, x)
            idx = np.linspace(0, c.n_x - 1, PROBE).astype(int)
            out[f"{name}/{seed}"] = {"obj": r.obj, "terms": r.terms, "grad_idx": idx.tolist(),
                                     "grad": r.grad[idx].tolist()}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(records(), f, indent=1, sort_keys=True)
    print("wrote", path)
