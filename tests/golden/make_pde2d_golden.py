"""Write fine-grid solutions of the 2-D steady transport equation for the
anisotropic model with drifts, in the two axisymmetric field geometries
(unipolar; reversing across a flat current sheet), each in both polarity
epochs: the reference of tests/test_oracle_pde2d.py.

Calls only oracle/ (and the seeded input descriptions); run from the
repository root:  python tests/golden/make_pde2d_golden.py
Output: tests/golden/pde2d_axisymmetric.json with, per case, the species,
the parameter set, the grid and J(T0) (Eq. 5 steady, with the estimator's
normalisation of Eq. 4: J = P0^2 f) at 0.3, 1 and 3 GeV/n seen from 1 AU,
30 deg north of the equator: protons in both geometries, He-4 and electrons
(the other species of the batched workload) with the unipolar field.
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


def params(sheet, polarity):
    # a 20 AU heliosphere with a shock at 14 AU: small enough for the oracle to run in seconds;
    # the flat sheet's minimum half-width is 4 deg (1 deg by default) for the same reason
    extra = dict(hcs_on=1.0, tilt_deg=0.0, dcs_min_deg=4.0) if sheet else dict(hcs_on=0.0)
    return W.params(R_out=20.0, R_ts=14.0, polarity=polarity, r0=OBSERVER[0], th0=OBSERVER[1], **extra)


UNIPOLAR_GRID = {"n_r": 160, "n_th": 180, "dlnP": 0.005, "P_top": 300.0, "th_stretch": 0.0}
SHEET_GRID = {"n_r": 120, "n_th": 240, "dlnP": 0.005, "P_top": 300.0, "th_stretch": 1.5}
CASES = [
    ("unipolar", "proton", False, UNIPOLAR_GRID),
    ("flat_sheet", "proton", True, SHEET_GRID),
    ("unipolar", "he4", False, UNIPOLAR_GRID),
    ("unipolar", "electron", False, UNIPOLAR_GRID),
]


def main():
    rec = {"T0": T0, "observer": OBSERVER, "cases": []}
    for name, species, sheet, grid in CASES:
        sp = W.SPECIES[species]
        P0 = [sp["A"] / abs(sp["Z"]) * math.sqrt(T * (T + 2 * sp["m0"])) for T in T0]
        for pol in (1.0, -1.0):
            t0 = time.time()
            p = params(sheet, pol)
            J = pde2d.solve(sp, p, OBSERVER[0], OBSERVER[1], P0, **grid)
            rec["cases"].append({"name": name, "species_name": species, "species": sp, "params": dict(p),
                                 "grid": grid, "J": [float(x) for x in J]})
            print(f"{name} {species} polarity {pol:+.0f}: J = {[float(x) for x in J]} ({time.time() - t0:.0f} s)",
                  flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "pde2d_axisymmetric.json"), "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
