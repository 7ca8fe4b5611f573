"""Write the Cartesian Monte Carlo solutions (oracle/sde_cartesian.c) that pin the
oracle's spherical step where the model depends on the longitude.

Calls only oracle/ (and the seeded input descriptions); run from the
repository root:  python tests/golden/make_cartesian_golden.py
Output: tests/golden/cartesian_tilted.json with, per case, J and its Monte
Carlo sigma (unbinned Eq. 4) at T0 = 0.3, 1, 3 GeV, the mean steps per path,
the paths per energy, the seed and the step scale.

Cases (the 20-AU heliosphere with a shock at 14 AU of the 2-D PDE pin, so
that the paths are short enough for many samples):
  * "validation": the four axisymmetric proton cases of
    tests/golden/pde2d_axisymmetric.json (unipolar field and flat current
    sheet, both polarity epochs), whose exact solutions the 2-D PDE gives --
    they pin this solver itself;
  * "tilted": the wavy current sheet (Sec. II.B), which no 2-D reduction
    covers: protons with a tilt of 30 deg and the standard rotation in both
    epochs, and with a tilt of 60 deg and a 100-day rotation (a slower spiral,
    where the longitude equation weighs more) in the A < 0 epoch, in which the
    sheet's drift carries positive particles; electrons (negative charge,
    beta ~ 1) with a tilt of 30 deg in the A > 0 epoch, in which it carries
    negative ones; He-4 (A/Z = 2) with a tilt of 30 deg in the A < 0 epoch.
Cases already in the output file are kept (the file is rewritten after every
case, so an interrupted run resumes where it stopped).
Every limit of the step rule is divided by 4 (step_scale 0.25), halving the
O(sqrt(dt)) bias of testing for the exit after each step.
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cartesian as CC  # noqa: E402
from paper_2502_06319_gb300 import workloads as W  # noqa: E402

STEP_SCALE = 0.25
SEED = 3


def tilted_cases(base):
    """(name, parameters, species) of the tilted-sheet cases."""
    P, E, H = W.PROTON, W.ELECTRON, W.HELIUM4
    return [("tilt30_A+", dict(base, hcs_on=1.0, tilt_deg=30.0, polarity=1.0), P),
            ("tilt30_A-", dict(base, hcs_on=1.0, tilt_deg=30.0, polarity=-1.0), P),
            ("tilt60_rot100_A-", dict(base, hcs_on=1.0, tilt_deg=60.0, polarity=-1.0, rot_period_day=100.0), P),
            ("tilt30_electron_A+", dict(base, hcs_on=1.0, tilt_deg=30.0, polarity=1.0), E),
            ("tilt30_he4_A-", dict(base, hcs_on=1.0, tilt_deg=30.0, polarity=-1.0), H)]


def main():
    CC.build()
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "pde2d_axisymmetric.json")))
    T0 = g["T0"]
    protons = [c for c in g["cases"] if c["species_name"] == "proton"]
    jobs = [("validation", f"{c['name']}_A{'+' if c['params']['polarity'] > 0 else '-'}", c["params"],
             c["species"], 8000) for c in protons]
    jobs += [("tilted", name, p, sp, 20000) for name, p, sp in tilted_cases(protons[0]["params"])]
    path = os.path.join(ROOT, "tests", "golden", "cartesian_tilted.json")
    out = {"T0": T0, "step_scale": STEP_SCALE, "seed": SEED, "cases": []}
    if os.path.exists(path):
        old = json.load(open(path))
        if (old["T0"], old["step_scale"], old["seed"]) == (T0, STEP_SCALE, SEED):
            out = old
    done = {c["name"] for c in out["cases"]}
    for kind, name, p, sp, n in jobs:
        if name in done:
            continue
        t0 = time.time()
        res = CC.run(p, sp, T0, [n] * len(T0), seed=SEED, step_scale=STEP_SCALE)
        J, S = CC.spectrum(res, sp, T0)
        rec = {"kind": kind, "name": name, "params": p, "species": sp, "n_per_energy": n, "J": J.tolist(),
               "sigma": S.tolist(), "mean_steps": float(res["steps"].mean()),
               "status_counts": np.bincount(res["status"], minlength=4).tolist(), "seconds": time.time() - t0}
        out["cases"].append(rec)
        print(kind, name, "J", J, "sigma_rel", S / J, "steps", rec["mean_steps"], "s", round(rec["seconds"]), flush=True)
        with open(path, "w") as f:
            json.dump(out, f)


if __name__ == "__main__":
    main()
