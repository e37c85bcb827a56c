"""Writes rt617_ttt_bounds.json: the lower bounds of Phi (eps = 0) that the time-to-target
comparison states its target against, for the held-out load profiles it uses.

For each profile (synth.load_profiles(rt617, 8, seed 5001), the generator the warm-start experiment
draws its held-out profiles from) it records the copper-plate bound of Sec. III-A and the
contingency-aware bound of oracle/copperplate.py (the copper plate plus the DC post-contingency
overloads of Sec. II-E, which are affine in the dispatch).  Calls only the oracle and the seeded
input generators.  Takes about 2 minutes per profile on 8 cores.

    python tests/golden/make_ttt_bounds.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle.copperplate import contingency_bound, copper_plate  # noqa: E402

SEED, COUNT = 5001, 8


def main():
    base = synth.rt617()
    prof = synth.load_profiles(base, COUNT, SEED)
    rows = []
    for i, lp in enumerate(prof):
        c = synth.with_loads(base, lp)
        t0 = time.time()
        cp = copper_plate(c)[0]
        cb, _, _, n_trip = contingency_bound(c)
        rows.append({"profile": i, "copper_plate": cp, "contingency_bound": cb, "triples": int(n_trip),
                     "seconds": round(time.time() - t0, 1)})
        print(rows[-1], flush=True)
    out = {"case": "rt617 (617 buses, 18 periods, 562 outages)",
           "profiles": f"synth.load_profiles(rt617, {COUNT}, seed {SEED})",
           "source": "oracle.copperplate.copper_plate (Sec. III-A) and contingency_bound (Sec. III-A plus the "
                     "DC contingency flows of Sec. II-E), both lower bounds of Phi at eps = 0",
           "rows": rows}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rt617_ttt_bounds.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
