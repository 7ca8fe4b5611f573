"""Write the FP64 oracle's full-size results for configs 1 and 2.

Calls only oracle/ (and the seeded input descriptions); run from the
repository root:  python tests/golden/make_golden.py
Output: tests/golden/oracle_c1.json, tests/golden/oracle_c2.json with, per
energy, the exit histogram (512 bins + under/overflow/failed), the binned
spectrum J and its sigma (Eq. 4), and the total step count.
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


def main():
    O.build()
    for name, job in (("c1", W.config1()), ("c2", W.config2())):
        t0 = time.time()
        out = O.job_run(job)
        H, J, S = O.job_spectrum(job, out)
        rec = {"config": name, "T_in": job.T_in, "n_per_energy": job.n_per_energy, "seed": job.seed,
               "bins": [job.bins.P_min, job.bins.P_max, job.bins.n],
               "hist": H.astype(np.int64).tolist(), "J": J.tolist(), "sigma": S.tolist(),
               "steps": int(out["steps"].astype(np.int64).sum()),
               "status_counts": np.bincount(out["status"], minlength=4).tolist(),
               "oracle_seconds": time.time() - t0, "threads": O.max_threads()}
        path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
        with open(path, "w") as f:
            json.dump(rec, f)
        print(name, "steps", rec["steps"], "seconds", round(rec["oracle_seconds"], 1), flush=True)


if __name__ == "__main__":
    main()
