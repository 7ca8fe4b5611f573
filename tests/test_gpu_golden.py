"""Full-size configs 1 and 2 against the FP64 oracle's stored results
(tests/golden/oracle_c*.json, written by tests/golden/make_golden.py, which
calls only the oracle).

FP64 path: every exit lands in the same bin, so the integer histograms are
equal exactly and the spectra to rounding.  Mixed path: per energy within 3
sigma of the combined Monte Carlo error and within 0.5 % relative."""
import json
import os

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import gpu_run, gpu_spectrum

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    with open(os.path.join(HERE, "golden", f"oracle_{name}.json")) as f:
        return json.load(f)


def _job(name, gold):
    """The workload with the golden file's stored inputs: the energies come from
    np.logspace, whose last bit may differ between machines."""
    job = W.config1() if name == "c1" else W.config2()
    assert np.allclose(job.T_in, gold["T_in"], rtol=1e-15, atol=0)
    assert job.n_per_energy == gold["n_per_energy"] and job.seed == gold.get("seed", job.seed)
    job.T_in = [float(t) for t in gold["T_in"]]
    return job


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_fp64_full_size_histogram_equals_oracle(name):
    gold = _golden(name)
    job = _job(name, gold)
    g, out, m = gpu_run(job, precision=cz.PREC_FP64)
    H, J, S = gpu_spectrum(job, out)
    m.close()
    assert int(g["steps"].astype(np.int64).sum()) == gold["steps"]
    assert np.array_equal(H.astype(np.int64), np.array(gold["hist"], dtype=np.int64))
    assert np.allclose(J, gold["J"], rtol=1e-12, atol=0) and np.allclose(S, gold["sigma"], rtol=1e-10, atol=0)


@pytest.mark.parametrize("precision", [cz.PREC_MIXED, cz.PREC_MIXED_F64ACC])
def test_mixed_config2_full_size_vs_oracle(precision):
    gold = _golden("c2")
    job = _job("c2", gold)
    g, out, m = gpu_run(job, precision=precision)
    H, J, S = gpu_spectrum(job, out)
    m.close()
    Jo, So = np.array(gold["J"]), np.array(gold["sigma"])
    rel = J / Jo - 1
    comb = np.hypot(S, So)
    print(f"config 2 precision {precision}: per-energy |rel| max {np.abs(rel).max():.2e}, "
          f"|dJ|/sigma max {np.max(np.abs(J - Jo) / comb):.2f}")
    assert np.all(np.abs(J - Jo) <= 3 * comb)
    assert np.all(np.abs(rel) <= 5e-3), rel
