"""Write the FP64 oracle's spectra for twelve items of the batched workload
(64 heliospheres x {p, He-4, e-} x 30 energies, counts 1e3-5e4).

Calls only oracle/ (and the seeded input descriptions); run from the
repository root:  python tests/golden/make_c3_golden.py
Output: tests/golden/oracle_c3_items.json.

The items are exact members of the batched workload (same parameter set,
species, energy, particle count, first particle identity and seed), so the
CUDA path's full-size run contains the very same quasi-particles.  Chosen to
span the workload's ranges: four heliospheres -- both polarity epochs (A > 0,
A < 0), each with a current-sheet tilt above 60 deg and one below 15 deg --
times the three species, at energies from 0.1 to 49 GeV/n, among the items
with at least 38 000 quasi-particles (so that the spectrum's relative Monte
Carlo error is ~0.1-0.3 %).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2502_06319_gb300 import workloads as W  # noqa: E402

# (parameter set, species, energy index): tilt 73 deg A > 0, 64 deg A < 0, 11 deg A < 0, 8 deg A > 0
PICK = ((11, "proton", 25), (11, "he4", 0), (11, "electron", 14),
        (2, "proton", 19), (2, "he4", 4), (2, "electron", 22),
        (6, "proton", 16), (6, "he4", 25), (6, "electron", 4),
        (30, "proton", 10), (30, "he4", 6), (30, "electron", 26))
SPECIES = ("proton", "he4", "electron")
NBINS = 512
MIN_N = 38000


def select(jobs, items):
    """(item index in the batched workload, job index, energy index) of the twelve items."""
    out = []
    n_e = len(jobs[0].T_in)
    for si, sp, e in PICK:
        j = 3 * si + SPECIES.index(sp)
        assert jobs[j].name == f"c3/{si}/{sp}"
        assert jobs[j].n_per_energy[e] >= MIN_N
        out.append((j * n_e + e, j, e))
    return out


def main():
    O.build()
    jobs = W.config3()
    params, species, items = W.items_of(jobs, 0)
    sel = select(jobs, items)
    prm_idx, sp_idx, T, pid, seed, owner = [], [], [], [], [], []
    for k, (ii, j, e) in enumerate(sel):
        pi, si, T_, n, fp, sd = items[ii]
        prm_idx += [pi] * n
        sp_idx += [si] * n
        T += [T_] * n
        pid += list(range(fp, fp + n))
        seed += [sd] * n
        owner += [k] * n
    t0 = time.time()
    out = O.run_particles(params, species, np.array(prm_idx), np.array(sp_idx), np.array(T),
                          np.array(pid, dtype=np.uint64), np.array(seed, dtype=np.uint64))
    secs = time.time() - t0
    out["energy"] = np.array(owner)
    H = O.histogram(out, len(sel), 0.1, 1000.0, NBINS)
    recs = []
    for k, (ii, j, e) in enumerate(sel):
        pi, si, T_, n, fp, sd = items[ii]
        Jk, Sk = O.spectrum_from_hist(H[k:k + 1], species[si], [T_], 0.1, 1000.0, NBINS)
        m = out["energy"] == k
        recs.append({"item": ii, "job": j, "energy_index": e, "param_idx": pi, "species_idx": si,
                     "set": PICK[k][0], "species": PICK[k][1], "T": T_, "n": n, "first_pid": fp,
                     "seed": sd, "tilt_deg": jobs[j].params["tilt_deg"], "polarity": jobs[j].params["polarity"],
                     "K0": jobs[j].params["K0"], "hist": H[k].astype(np.int64).tolist(),
                     "J": float(Jk[0]), "sigma": float(Sk[0]),
                     "steps": int(out["steps"][m].astype(np.int64).sum()),
                     "status_counts": np.bincount(out["status"][m], minlength=4).tolist()})
        print(f"item {ii}: set {PICK[k][0]} {PICK[k][1]} T {T_:.3g} n {n}: J {Jk[0]:.6g} "
              f"sigma_rel {Sk[0] / Jk[0]:.4f}", flush=True)
    rec = {"workload": "batched: 64 heliospheres x {p, He-4, e-} x 30 energies (seeds 20250210/20250211)",
           "bins": [0.1, 1000.0, NBINS], "items": recs, "oracle_seconds": secs, "threads": O.max_threads()}
    with open(os.path.join(ROOT, "tests", "golden", "oracle_c3_items.json"), "w") as f:
        json.dump(rec, f)
    print("steps", int(out["steps"].astype(np.int64).sum()), "seconds", round(secs, 1))


if __name__ == "__main__":
    main()
