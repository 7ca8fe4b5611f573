"""Radial shells of the inner heliosphere (Sec. II.B) on the GPU, through the C ABI.

FP64: paths through 15 shells of a synthetic solar-cycle heliosphere equal the
oracle's bit for bit, coefficients inside the blend windows are bit-identical,
and constant tables reproduce the single-region model.  Mixed: spectra within
3 sigma and 0.5 % of the oracle; a batch mixing shell and single-region
parameter sets (one launch of the shell variant of the kernel) gives every
item exactly as the same set alone.
"""
import math

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import compare_paths, gpu_run, gpu_spectrum, torch

pytestmark = pytest.mark.gpu

SER = W.solar_cycle_series()
SHELLS = W.shell_params(SER, rotation=60, max_steps=2_000_000)


def test_fp64_shell_paths_equal_oracle(orc):
    job = W.Job(SHELLS, W.PROTON, [0.2, 2.0, 20.0], [60, 40, 8], seed=41)
    g, out, m = gpu_run(job, precision=cz.PREC_FP64)
    m.close()
    o = orc.job_run(job)
    same, worst = compare_paths(g, o)
    assert same == 1.0 and worst <= 1e-10, (same, worst)


def test_fp64_coefficients_in_blend_windows_bit_identical(orc):
    t = torch()
    dR = 85.0 / 15
    rng = np.random.default_rng(5)
    st = []
    for e in range(1, 15):
        for x in (-0.45, -0.2, 0.0, 0.1, 0.33, 0.49):
            st.append((e * dR + x, rng.uniform(0.2, math.pi - 0.2), rng.uniform(0, 2 * math.pi),
                       rng.uniform(-1.0, 5.0)))
    st = np.array(st)
    for prec in (0, 1):
        m = cz.Model(cz.make_params(SHELLS))
        outd = t.empty(st.shape[0] * cz.DEBUG_EVAL_N, dtype=t.float64, device="cuda")
        cz.cosmica_debug_eval(m.h, cz.make_species(W.HELIUM4), prec, t.as_tensor(st).cuda(), outd)
        t.cuda.synchronize()
        m.close()
        got = outd.cpu().numpy().reshape(st.shape[0], cz.DEBUG_EVAL_N)
        for i in range(st.shape[0]):
            ref = orc.evaluate(SHELLS, W.HELIUM4, *st[i])
            for j, name in enumerate(cz.DEBUG_EVAL_NAMES):
                a, b = got[i, j], ref[name]
                if prec == 0:
                    assert a == b or (np.isnan(a) and np.isnan(b)), (i, name, a, b)
                elif name in ("Kpar", "Krr", "Ktt", "Kpp"):
                    assert abs(a - b) <= 1e-4 * abs(b), (i, name, a, b)   # the blended K0 in FP32


def test_fp64_constant_tables_reproduce_single_region():
    p1 = W.params(R_ts=85.0, R_out=122.0, K0=14.0, tilt_deg=30.0, max_steps=2_000_000)
    p2 = dict(p1, n_shells=15.0, shell_K0=(14.0,) * 15, shell_tilt_deg=(30.0,) * 15)
    T, N = [0.3, 3.0], [80, 80]
    a, _, m1 = gpu_run(W.Job(p1, W.PROTON, T, N, seed=2), precision=cz.PREC_FP64)
    b, _, m2 = gpu_run(W.Job(p2, W.PROTON, T, N, seed=2), precision=cz.PREC_FP64)
    m1.close()
    m2.close()
    for k in ("r", "th", "ph", "lnP", "s", "steps", "status"):
        assert np.array_equal(a[k], b[k]), k


def test_mixed_shell_spectrum_vs_oracle(orc):
    job = W.Job(SHELLS, W.PROTON, [0.3, 3.0, 30.0], [5000, 5000, 5000], seed=43,
                bins=W.Bins(0.1, 1000.0, 512))
    g, out, m = gpu_run(job, precision=cz.PREC_MIXED)
    H, J, S = gpu_spectrum(job, out)
    m.close()
    o = orc.job_run(job)
    Ho, Jo, So = orc.job_spectrum(job, o)
    rel = J / Jo - 1
    comb = np.hypot(S, So)
    print("shells mixed vs oracle rel per energy:", np.round(rel, 4), "sigma_rel:", np.round(So / Jo, 4))
    assert np.all(np.abs(J - Jo) <= 3 * comb)
    assert np.all(np.abs(rel) <= 5e-3), rel


@pytest.mark.parametrize("precision", [cz.PREC_MIXED, cz.PREC_MIXED_F64ACC])
def test_batch_mixing_shell_and_single_region_sets(precision):
    t = torch()
    single = W.params(R_ts=85.0, R_out=122.0, K0=12.0, tilt_deg=40.0, max_steps=2_000_000)
    sets = [SHELLS, single]
    items = [(0, 0, 0.4, 70, 0, 5), (1, 0, 0.4, 70, 70, 5), (0, 0, 4.0, 33, 140, 5), (1, 0, 4.0, 45, 173, 5)]
    b = cz.cosmica_batch_create([cz.make_params(p, precision) for p in sets], [cz.make_species(W.PROTON)])
    out = cz.ExitBuffers(sum(i[3] for i in items))
    cz.cosmica_batch_run(b, cz.make_items(items), len(items), out)
    t.cuda.synchronize()
    g = out.numpy()
    cz.cosmica_batch_destroy(b)
    off = 0
    for (pi, si, T_, n, fp, sd) in items:
        one = cz.cosmica_batch_create([cz.make_params(sets[pi], precision)], [cz.make_species(W.PROTON)])
        o1 = cz.ExitBuffers(n)
        cz.cosmica_batch_run(one, cz.make_items([(0, 0, T_, n, fp, sd)]), 1, o1)
        t.cuda.synchronize()
        s = o1.numpy()
        cz.cosmica_batch_destroy(one)
        for key in ("r", "th", "ph", "lnP", "s", "steps", "status"):
            assert np.array_equal(g[key][off:off + n], s[key]), (pi, T_, key)
        off += n


def test_invalid_shell_tables_are_rejected():
    for bad in (dict(n_shells=17.0), dict(n_shells=15.0, shell_blend_AU=3.0),
                dict(n_shells=15.0, shell_K0=(0.0,) * 15), dict(n_shells=15.0, shell_tilt_deg=(95.0,) * 15)):
        p = dict(SHELLS, **bad)
        with pytest.raises(cz.CosmicaError):
            cz.Model(cz.make_params(p))
