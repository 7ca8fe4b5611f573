"""Nose-squashed heliosphere (Sec. II.B) on the GPU, through the C ABI.

FP64: paths through the squashed shock to the squashed outer boundary equal
the oracle's bit for bit, and the coefficients next to the shock surface are
bit-identical (the drift gains d/dphi terms there).  Mixed: spectra within
3 sigma and 0.5 % of the oracle, and a batch mixing squashed and spherical
parameter sets gives every item exactly as the same set alone.
"""
import math

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import compare_paths, gpu_run, gpu_spectrum, torch

pytestmark = pytest.mark.gpu

SQ = W.params(R_ts=85.0, R_out=122.0, max_steps=2_000_000, **W.SQUASHED)


def test_fp64_squashed_paths_equal_oracle(orc):
    job = W.Job(SQ, W.PROTON, [0.2, 2.0, 20.0], [60, 40, 8], seed=51)
    g, out, m = gpu_run(job, precision=cz.PREC_FP64)
    m.close()
    o = orc.job_run(job)
    same, worst = compare_paths(g, o)
    assert same == 1.0 and worst <= 1e-10, (same, worst)


def test_coefficients_next_to_the_squashed_shock(orc):
    t = torch()
    rng = np.random.default_rng(9)
    n = np.array([math.sin(SQ["nose_th"]) * math.cos(SQ["nose_ph"]),
                  math.sin(SQ["nose_th"]) * math.sin(SQ["nose_ph"]), math.cos(SQ["nose_th"])])
    st = []
    for _ in range(120):
        th, ph = rng.uniform(0.2, math.pi - 0.2), rng.uniform(0, 2 * math.pi)
        d = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        mu = float(d @ n)
        a, b, c = 85.0 * 2.35 / 2, 85.0 * 1.15, 85.0 * 0.35 / 2
        A = mu * mu / a ** 2 + (1 - mu * mu) / b ** 2
        B = mu * c / a ** 2
        R = (-B + math.sqrt(B * B - A * (c * c / a ** 2 - 1))) / A
        st.append((R + rng.uniform(-2.0, 2.0), th, ph, rng.uniform(-1.0, 5.0)))
    st = np.array(st)
    for prec in (0, 1):
        m = cz.Model(cz.make_params(SQ))
        outd = t.empty(st.shape[0] * cz.DEBUG_EVAL_N, dtype=t.float64, device="cuda")
        cz.cosmica_debug_eval(m.h, cz.make_species(W.PROTON), prec, t.as_tensor(st).cuda(), outd)
        t.cuda.synchronize()
        m.close()
        got = outd.cpu().numpy().reshape(st.shape[0], cz.DEBUG_EVAL_N)
        for i in range(st.shape[0]):
            ref = orc.evaluate(SQ, W.PROTON, *st[i])
            for j, name in enumerate(cz.DEBUG_EVAL_NAMES):
                a, b = got[i, j], ref[name]
                if prec == 0:
                    assert a == b or (np.isnan(a) and np.isnan(b)), (i, name, a, b)
                elif name in ("Kpar", "Krr", "Ktt", "Kpp", "Ar"):
                    # the shock's position along the point's direction, in FP32
                    assert abs(a - b) <= 2e-3 * abs(b) + 1e-6 * ref["Kpar"], (i, name, a, b)


def test_mixed_squashed_spectrum_vs_oracle(orc):
    job = W.Job(SQ, W.PROTON, [0.3, 3.0, 30.0], [5000, 5000, 5000], seed=53, bins=W.Bins(0.1, 1000.0, 512))
    g, out, m = gpu_run(job, precision=cz.PREC_MIXED)
    H, J, S = gpu_spectrum(job, out)
    m.close()
    o = orc.job_run(job)
    Ho, Jo, So = orc.job_spectrum(job, o)
    rel = J / Jo - 1
    comb = np.hypot(S, So)
    print("squashed mixed vs oracle rel per energy:", np.round(rel, 4), "sigma_rel:", np.round(So / Jo, 4))
    assert np.all(np.abs(J - Jo) <= 3 * comb)
    assert np.all(np.abs(rel) <= 5e-3), rel


def test_batch_mixing_squashed_and_spherical_sets():
    t = torch()
    sph = W.params(R_ts=85.0, R_out=122.0, max_steps=2_000_000)
    sets = [SQ, sph]
    items = [(0, 0, 0.4, 64, 0, 3), (1, 0, 0.4, 64, 64, 3), (0, 0, 4.0, 40, 128, 3), (1, 0, 4.0, 21, 168, 3)]
    b = cz.cosmica_batch_create([cz.make_params(p, cz.PREC_MIXED) for p in sets], [cz.make_species(W.PROTON)])
    out = cz.ExitBuffers(sum(i[3] for i in items))
    cz.cosmica_batch_run(b, cz.make_items(items), len(items), out)
    t.cuda.synchronize()
    g = out.numpy()
    cz.cosmica_batch_destroy(b)
    off = 0
    for (pi, si, T_, n, fp, sd) in items:
        one = cz.cosmica_batch_create([cz.make_params(sets[pi], cz.PREC_MIXED)], [cz.make_species(W.PROTON)])
        o1 = cz.ExitBuffers(n)
        cz.cosmica_batch_run(one, cz.make_items([(0, 0, T_, n, fp, sd)]), 1, o1)
        t.cuda.synchronize()
        s = o1.numpy()
        cz.cosmica_batch_destroy(one)
        for key in ("r", "th", "ph", "lnP", "s", "steps", "status"):
            assert np.array_equal(g[key][off:off + n], s[key]), (pi, T_, key)
        off += n


def test_start_outside_the_squashed_boundary_is_rejected():
    # 125 AU toward the tail lies inside (tail at 195 AU); toward the nose it is outside
    p_in = dict(SQ, r0=125.0, th0=math.pi - SQ["nose_th"], ph0=(SQ["nose_ph"] + math.pi) % (2 * math.pi))
    cz.Model(cz.make_params(p_in)).close()
    p_out = dict(SQ, r0=125.0, th0=SQ["nose_th"], ph0=SQ["nose_ph"])
    with pytest.raises(cz.CosmicaError):
        cz.Model(cz.make_params(p_out))
