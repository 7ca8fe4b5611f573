"""Mixed precision (FP32 coefficients and normals, compensated FP32 or FP64
accumulation, exact boundary test) against the FP64 references.

Mixed paths use their own FP32 uniforms from the same Philox words, so they are
paired with the FP64 paths (same particle identities); the spectra are
compared per energy: within 3 sigma of the combined Monte Carlo error and
within 0.5 % relative."""
import math

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import gpu_run, gpu_spectrum, torch

pytestmark = pytest.mark.gpu

ACCS = [cz.PREC_MIXED, cz.PREC_MIXED_F64ACC]


@pytest.mark.parametrize("acc", ACCS)
def test_mixed_config0_vs_oracle(orc, acc):
    job = W.config0()
    g, out, m = gpu_run(job, precision=acc)
    assert np.all(g["status"] == cz.PATH_EXIT)
    o = orc.job_run(job)
    H, J, S = gpu_spectrum(job, out)
    Ho, Jo, So = orc.job_spectrum(job, o)
    comb = math.hypot(S[0], So[0])
    rel = abs(J[0] / Jo[0] - 1)
    print(f"config0 acc={acc}: J={J[0]:.6g} oracle={Jo[0]:.6g} rel={rel:.2e} sigma_rel={S[0] / J[0]:.2e}")
    assert abs(J[0] - Jo[0]) <= 3 * comb and rel <= 5e-3
    # smooth isotropic paths stay paired with the FP64 paths
    same = (g["steps"] == o["steps"]).mean()
    assert same > 0.9, same
    m.close()


@pytest.mark.parametrize("acc", ACCS)
def test_mixed_full_model_vs_oracle(orc, acc):
    T = W.logspace(0.1, 100.0, 10)
    job = W.Job(W.params(), W.PROTON, T, [300] * 10, seed=21, bins=W.Bins(0.1, 1000.0, 512))
    g, out, m = gpu_run(job, precision=acc)
    o = orc.job_run(job)
    H, J, S = gpu_spectrum(job, out)
    Ho, Jo, So = orc.job_spectrum(job, o)
    comb = np.hypot(S, So)
    print("full model acc=%d rel err per energy:" % acc, np.round(J / Jo - 1, 4).tolist())
    assert np.all(np.abs(J - Jo) <= 3 * comb), (J, Jo, comb)
    m.close()
