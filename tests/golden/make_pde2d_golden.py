"""Write fine-grid solutions of the 2-D steady transport equation for the
full anisotropic model without a current sheet (unipolar field, both
polarities), the reference of tests/test_oracle_pde2d.py.

Calls only oracle/ (and the seeded input descriptions); run from the
repository root:  python tests/golden/make_pde2d_golden.py
Output: tests/golden/pde2d_unipolar.json with the parameter set, the observer,
the energies, the grid and J(T0) per polarity (Eq. 5 steady, with the
estimator's normalisation of Eq. 4: J = P0^2 f).
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pde2d  # noqa: E402
from paper_2502_06319_gb300 import workloads as W  # noqa: E402

T0 = [0.3, 1.0, 3.0]
OBSERVER = (1.0, math.pi / 3)
GRID = {"n_r": 160, "n_th": 180, "dlnP": 0.005, "P_top": 300.0}


def params(polarity):
    # a 20 AU heliosphere with a shock at 14 AU: small enough for the oracle to run in seconds
    return W.params(R_out=20.0, R_ts=14.0, hcs_on=0.0, polarity=polarity, r0=OBSERVER[0], th0=OBSERVER[1])


def main():
    sp = W.PROTON
    P0 = [sp["A"] / abs(sp["Z"]) * math.sqrt(T * (T + 2 * sp["m0"])) for T in T0]
    rec = {"species": sp, "T0": T0, "observer": OBSERVER, "grid": GRID, "cases": []}
    for pol in (1.0, -1.0):
        t0 = time.time()
        p = params(pol)
        J = pde2d.solve(sp, p, OBSERVER[0], OBSERVER[1], P0, **GRID)
        rec["cases"].append({"params": {k: v for k, v in p.items()}, "J": [float(x) for x in J]})
        print(f"polarity {pol:+.0f}: J = {list(J)} ({time.time() - t0:.0f} s)")
    with open(os.path.join(ROOT, "tests", "golden", "pde2d_unipolar.json"), "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
