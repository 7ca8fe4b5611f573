"""The CUDA path against the independent 2-D PDE solution of the axisymmetric
model with drifts (unipolar field: protons, He-4 and electrons; flat current
sheet: protons; both polarity epochs each), through the C ABI: mixed-precision
spectra (Eq. 4, unbinned) within 3 sigma plus 0.5 % of the stored fine-grid
solutions of the steady transport equation (Eq. 5), the same bar the FP64
oracle meets in test_oracle_pde2d.py.  He-4 (A/Z = 2) and electrons (negative
charge, beta ~ 1) check the species-dependent parts of the mixed step: the
rigidity of a kinetic energy per nucleon, beta, and the sign of the drift.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import gpu_run, gpu_unbinned

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pde2d_axisymmetric.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("k", range(8))
@pytest.mark.parametrize("precision", [cz.PREC_MIXED, cz.PREC_MIXED_F64ACC], ids=["mixed", "f64acc"])
def test_mixed_spectrum_matches_pde(k, precision):
    g = _golden()
    case = g["cases"][k]
    job = W.Job(case["params"], case["species"], list(g["T0"]), [20000] * len(g["T0"]), seed=77)
    res, out, m = gpu_run(job, precision=precision)
    m.close()
    assert np.all(res["status"] == 1), np.bincount(res["status"])
    J, S = gpu_unbinned(job, out, 0)
    Jp = np.array(case["J"])
    assert np.all(np.abs(J - Jp) < 3.0 * S + 0.005 * Jp), (case["name"], case["species_name"],
                                                           case["params"]["polarity"], J, Jp, S)
