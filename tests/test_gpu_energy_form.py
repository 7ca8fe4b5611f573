"""The energy formulation (Eq. 1: kinetic energy integrated with
A_T = (2/3)(V/r) alpha T, loss L = (2V/(3r))(1 + beta^2) accumulated for the
weight of Eq. 4) on the GPU, against the oracle's energy formulation, and the
loss-weighted spectrum against the momentum form's."""
import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import compare_paths, gpu_run, gpu_unbinned

pytestmark = pytest.mark.gpu


def _energy(p):
    return dict(p, formulation=1.0)


@pytest.mark.parametrize("model", ["iso", "full"])
def test_fp64_energy_form_paths_and_weights_bit_identical(orc, model):
    base = W.config0().params if model == "iso" else W.params()
    job = W.Job(_energy(dict(base, dt_fixed=0.02) if model == "iso" else _energy(base)), W.PROTON,
                [0.2, 2.0, 20.0], [40, 41, 39], seed=77)
    g, out, m = gpu_run(job, precision=cz.PREC_FP64, with_lw=True)
    o = orc.job_run(job)
    frac, worst = compare_paths(g, o)
    assert frac >= 0.999 and worst <= 1e-10, (frac, worst)
    same = g["steps"] == o["steps"]
    assert np.array_equal(g["lw"][same], o["lw"][same])
    J, S = gpu_unbinned(job, out, 1)
    Jo, So = orc.spectrum_energy_form(o, job.species, job.T_in)
    assert np.allclose(J, Jo, rtol=1e-12, atol=0) and np.allclose(S, So, rtol=1e-10, atol=0)
    m.close()


def test_unbinned_momentum_spectrum_matches_oracle(orc):
    job = W.Job(W.params(), W.HELIUM4, [0.3, 3.0], [60, 60], seed=78)
    g, out, m = gpu_run(job, precision=cz.PREC_FP64)
    o = orc.job_run(job)
    J, S = gpu_unbinned(job, out, 0)
    Jo, So = orc.spectrum_unbinned(o, job.species, job.T_in)
    assert np.allclose(J, Jo, rtol=1e-12, atol=0) and np.allclose(S, So, rtol=1e-10, atol=0)
    m.close()


@pytest.mark.parametrize("precision", [cz.PREC_MIXED, cz.PREC_MIXED_F64ACC])
def test_mixed_energy_form_matches_momentum_form(orc, precision):
    """Same physics by two formulations on the GPU, and the energy form against the oracle's."""
    T = W.logspace(0.2, 50.0, 6)
    p = W.params()
    mom = W.Job(p, W.PROTON, T, [3000] * 6, seed=79)
    en = W.Job(_energy(p), W.PROTON, T, [3000] * 6, seed=79)
    gm, outm, mm = gpu_run(mom, precision=precision, with_lw=True)
    ge, oute, me = gpu_run(en, precision=precision, with_lw=True)
    Jm, Sm = gpu_unbinned(mom, outm, 0)
    Je, Se = gpu_unbinned(en, oute, 1)
    print(f"precision {precision}: energy/momentum - 1 =", np.round(Je / Jm - 1, 4).tolist())
    assert np.all(np.abs(Je - Jm) <= 3 * np.hypot(Sm, Se) + 2e-3 * Jm)
    assert np.all(gm["lw"] == 0.0) and np.all(ge["lw"] < 0.0)
    small = W.Job(_energy(p), W.PROTON, T, [150] * 6, seed=79)
    o = orc.job_run(small)
    Jo, So = orc.spectrum_energy_form(o, small.species, small.T_in)
    gs, outs, ms = gpu_run(small, precision=precision, with_lw=True)
    Js, Ss = gpu_unbinned(small, outs, 1)
    assert np.all(np.abs(Js - Jo) <= 3 * np.hypot(Ss, So)), (Js, Jo)
    for mm_ in (mm, me, ms):
        mm_.close()


def test_energy_form_needs_weights_and_is_rejected_by_the_server():
    job = W.Job(_energy(W.params()), W.PROTON, [1.0], [10], seed=1)
    with pytest.raises(cz.CosmicaError) as e:
        gpu_run(job, precision=cz.PREC_MIXED, with_lw=False)
    assert e.value.status == cz.ERR_INVALID
    srv = cz.cosmica_server_create(1 << 30, cz.PREC_MIXED)
    req = cz.Request(cz.make_params(_energy(W.params()), cz.PREC_MIXED), cz.make_species(W.PROTON), [1.0], [10], 1,
                     cz.make_bins(0.1, 1000.0, 64))
    with pytest.raises(cz.CosmicaError):
        cz.cosmica_server_submit(srv, req)
    cz.cosmica_server_destroy(srv)
