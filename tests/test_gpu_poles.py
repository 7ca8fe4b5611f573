"""Paths at the poles in the mixed path.

The SFU sine has an absolute error bound, so at theta ~ 1e-7 it can return 0 and
1/sin(theta) becomes infinite; the mixed step therefore takes sin(theta) from the
compensated state's distance to the nearer pole (Taylor series below 0.1 rad),
and folds theta at pi on the full float-float value.  Config 3 at full size
exercises this ~15 000 times (every path must exit); here it is checked directly:
coefficients next to both poles are finite and agree with the FP64 oracle, and
paths started next to a pole all exit with spectra that agree with the oracle.
"""
import math

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import gpu_run, gpu_spectrum, torch

pytestmark = pytest.mark.gpu


def test_mixed_coefficients_next_to_the_poles(orc):
    t = torch()
    p = W.params(R_ts=85.0, R_out=122.0, tilt_deg=71.0)
    st = []
    for th in (1e-9, 6e-8, 1.8e-7, 1e-6, 3e-4, math.pi - 3e-8, math.pi - 2e-7, math.pi - 1e-5):
        for r, ph, lnP in ((1.5, 0.4, -0.5), (40.0, 2.5, 0.3), (107.0, 5.3, -0.1)):
            st.append((r, th, ph, lnP))
    st = np.array(st)
    m = cz.Model(cz.make_params(p))
    out = t.empty(st.shape[0] * cz.DEBUG_EVAL_N, dtype=t.float64, device="cuda")
    cz.cosmica_debug_eval(m.h, cz.make_species(W.PROTON), cz.PREC_MIXED, t.as_tensor(st).cuda(), out)
    t.cuda.synchronize()
    m.close()
    got = out.cpu().numpy().reshape(st.shape[0], cz.DEBUG_EVAL_N)
    assert np.all(np.isfinite(got))
    for i in range(st.shape[0]):
        ref = orc.evaluate(p, W.PROTON, *st[i])
        for name in ("Ath", "Aph", "Kpar", "dt"):
            a, b = got[i, cz.DEBUG_EVAL_NAMES.index(name)], ref[name]
            assert abs(a - b) <= 2e-3 * abs(b) + 1e-12, (st[i], name, a, b)


@pytest.mark.parametrize("th0", [1e-6, math.pi - 1e-6])
def test_mixed_paths_started_at_a_pole(orc, th0):
    p = W.params(R_ts=85.0, R_out=122.0, tilt_deg=71.0, th0=th0, max_steps=2_000_000)
    job = W.Job(p, W.PROTON, [0.15, 2.0], [1500, 1500], seed=61, bins=W.Bins(0.1, 1000.0, 512))
    g, out, m = gpu_run(job, precision=cz.PREC_MIXED)
    H, J, S = gpu_spectrum(job, out)
    m.close()
    assert np.all(g["status"] == cz.PATH_EXIT), np.unique(g["status"], return_counts=True)
    o = orc.job_run(job)
    Ho, Jo, So = orc.job_spectrum(job, o)
    assert np.all(np.abs(J - Jo) <= 3 * np.hypot(S, So)), (J, Jo, S, So)
