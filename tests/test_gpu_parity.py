"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

FP64 mode (-fmad=false, deterministic elementary functions): at least 99.9 %
of paths exit on the same step as the oracle with the exit state within 1e-10
relative; histograms are integer and must match exactly; spectra agree to
1e-12.  Mixed mode: spectra agree within 3 sigma of the Monte Carlo error and
0.5 % (see test_gpu_mixed.py).
"""
import math
import zlib

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import compare_paths, gpu_run, gpu_spectrum, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    t = torch()
    if not t.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cz.lib()


def _dev(a, dtype=None):
    t = torch()
    return t.as_tensor(a, dtype=dtype).cuda()


# ------------------------------------------------------------- RNG pieces --
def test_philox_bit_exact_vs_oracle(orc):
    t = torch()
    rng = np.random.default_rng(0)
    for key in ((1, 0), (0xDEADBEEF, 0x01234567), (0xFFFFFFFF, 0xFFFFFFFF)):
        ctr = rng.integers(0, 2**32, size=(340_000, 4), dtype=np.uint64).astype(np.uint32)   # > 10^6 counters in all
        ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [7, 0, 0, 0]]
        d_ctr = _dev(ctr.view(np.int32))
        d_out = t.empty_like(d_ctr)
        cz.cosmica_debug_philox(d_ctr, key[0], key[1], d_out)
        t.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, orc.philox(ctr, key))


def test_philox_bit_exact_vs_curand(orc):
    """cuRAND's Philox4_32_10 after curand_init(seed, subsequence, offset = 4n) returns
    the block for counter (n_lo, n_hi, sub_lo, sub_hi), key (seed_lo, seed_hi)."""
    t = torch()
    rng = np.random.default_rng(1)
    n = 50_000
    sub = rng.integers(0, 2**40, size=n, dtype=np.uint64)
    blk = rng.integers(0, 2**34, size=n, dtype=np.uint64)
    seed = 0x0123456789ABCDEF
    d_sub = _dev(sub.view(np.int64))
    d_off = _dev((blk * np.uint64(4)).view(np.int64))
    d_out = t.empty(4 * n, dtype=t.int32, device="cuda")
    cz.cosmica_debug_curand_philox(seed, d_sub, d_off, d_out)
    t.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint32).reshape(n, 4)
    ctr = np.stack([blk & np.uint64(0xFFFFFFFF), blk >> np.uint64(32),
                    sub & np.uint64(0xFFFFFFFF), sub >> np.uint64(32)], axis=1).astype(np.uint32)
    ref = orc.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    assert np.array_equal(got, ref)


def test_fp64_elementary_functions_bit_identical(orc):
    t = torch()
    rng = np.random.default_rng(2)
    cases = {"exp": rng.uniform(-40, 12, 300_000), "log": np.exp(rng.uniform(-25, 10, 300_000)),
             "sin": rng.uniform(-10, 400, 300_000), "cos": rng.uniform(-10, 400, 300_000),
             "tanh": rng.uniform(-25, 25, 300_000), "atan": rng.uniform(-8, 8, 300_000)}
    for name, x in cases.items():
        dx = _dev(x)
        dy = t.empty_like(dx)
        cz.cosmica_debug_fn64(name, dx, dy)
        t.cuda.synchronize()
        got = dy.cpu().numpy()
        ref = orc.fn(name, x)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), name


def test_fp64_normals_bit_identical(orc):
    t = torch()
    for seed, pid0, step in ((1, 0, 0), (12345, 10**12, 77), (2**63 + 5, 2**40, 4_000_000)):
        n = 100_000
        z = t.empty(3 * n, dtype=t.float64, device="cuda")
        cz.cosmica_debug_normals64(seed, pid0, n, step, z)
        t.cuda.synchronize()
        assert np.array_equal(z.cpu().numpy().reshape(n, 3), orc.normals(seed, pid0, n, step))



def test_fp32_normals_within_their_error_bound(orc):
    """The mixed step's normals (FP32, SFU approximations) against Box-Muller in FP64 on the
    same Philox words.  The words must be the oracle's block for (seed, pid, step); each word
    maps to u = ((x >> 9) + 1/2) 2^-23, and z0 = rho0 cos(2 pi u1), z1 = rho0 sin(2 pi u1),
    z2 = rho2 cos(2 pi u3), rho = sqrt(-2 ln u) -- the pairing of the FP64 step, so that mixed
    and FP64 paths draw the same noise.  The bound is built from the documented maximum errors
    of the approximations used: __logf 2^-21.41 absolute on [0.5, 2] and 3 ulp elsewhere,
    __sincosf 2^-21.41 absolute on [-pi, pi], the approximate square root 3 ulp, the rounded
    angle 2 pi u - pi (FP32 constants and one fma), with a factor 4 of margin."""
    t = torch()
    for seed, pid0, step in ((1, 0, 0), (2**63 + 5, 2**40 - 3, 4_000_000)):
        n = 1 << 20
        z = t.empty(3 * n, dtype=t.float32, device="cuda")
        w = t.empty(4 * n, dtype=t.int32, device="cuda")
        cz.cosmica_debug_normals32(seed, pid0, n, step, z, w)
        t.cuda.synchronize()
        z = z.cpu().numpy().reshape(n, 3).astype(np.float64)
        w = w.cpu().numpy().view(np.uint32).reshape(n, 4)
        pid = np.arange(pid0, pid0 + n, dtype=np.uint64)
        ctr = np.stack([np.full(n, step, np.uint64), pid & 0xFFFFFFFF, pid >> np.uint64(32),
                        np.zeros(n, np.uint64)], axis=1).astype(np.uint32)
        assert np.array_equal(w, orc.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32)))
        u = ((w >> 9).astype(np.float64) + 0.5) * 2.0**-23
        rho0, rho2 = np.sqrt(-2.0 * np.log(u[:, 0])), np.sqrt(-2.0 * np.log(u[:, 2]))
        ref = np.stack([rho0 * np.cos(2 * np.pi * u[:, 1]), rho0 * np.sin(2 * np.pi * u[:, 1]),
                        rho2 * np.cos(2 * np.pi * u[:, 3])], axis=1)
        rho = np.stack([rho0, rho0, rho2], axis=1)
        lnu = np.stack([np.log(u[:, 0])] * 2 + [np.log(u[:, 2])], axis=1)
        e_ln = 2.0**-21.41 * np.maximum(1.0, np.abs(lnu))      # error of ln u
        d_rho = np.minimum(np.sqrt(2.0 * e_ln), 2.0 * e_ln / rho) + 3.0 * 2.0**-23 * rho
        d_ang = 2.0**-21.41 + 4.0e-7                             # sincos + rounded angle
        tol = 4.0 * (d_rho + rho * d_ang + 2.0**-24 * np.abs(ref))
        err = np.abs(z - ref)
        assert np.all(err <= tol), (float((err / tol).max()), np.unravel_index(np.argmax(err / tol), err.shape))
        assert abs(z.mean()) < 5.0 / np.sqrt(z.size) and abs(z.var() - 1.0) < 0.01
        # paired with the FP64 step's normals (whose uniforms keep all 32 bits)
        z64 = orc.normals(seed, pid0, n, step)
        for c in range(3):
            assert np.corrcoef(z[:, c], z64[:, c])[0, 1] > 0.99999

# ------------------------------------------------------------ coefficients --
_ORACLE_NAMES = {"V": "V", "Gam": "Gam", "Kpar": "Kpar", "Krr": "Krr", "Ktt": "Ktt", "Kpp": "Kpp",
                 "Krp": "Krp", "Ar": "Ar", "Ath": "Ath", "Aph": "Aph", "L00": "L00", "L11": "L11",
                 "L20": "L20", "L22": "L22", "h": "h", "delta_cs": "delta_cs", "vdr": "vdr", "vdth": "vdth",
                 "vdph": "vdph", "dlnP": "dlnP", "dt": "dt"}

MODELS = {
    "c0": W.config0().params,
    "full": W.params(),
    "ts_tilt60": W.params(R_ts=85.0, R_out=122.0, tilt_deg=60.0, polarity=-1.0),
    "unipolar": W.params(hcs_on=0.0),
    "nodrift": W.params(drift_on=0.0),
    "shells": W.shell_params(W.solar_cycle_series(), rotation=60),
}


def _states(n, rng):
    r = np.exp(rng.uniform(math.log(0.1), math.log(121.0), n))
    th = rng.uniform(0.01, math.pi - 0.01, n)
    ph = rng.uniform(0, 2 * math.pi, n)
    lnP = rng.uniform(-1.5, 6.0, n)
    return np.stack([r, th, ph, lnP], axis=1)


def _gpu_eval(params, species, prec, st):
    t = torch()
    m = cz.Model(cz.make_params(params))
    out = t.empty(st.shape[0] * cz.DEBUG_EVAL_N, dtype=t.float64, device="cuda")
    cz.cosmica_debug_eval(m.h, cz.make_species(species), prec, _dev(st), out)
    t.cuda.synchronize()
    m.close()
    return out.cpu().numpy().reshape(st.shape[0], cz.DEBUG_EVAL_N)


@pytest.mark.parametrize("model", list(MODELS))
@pytest.mark.parametrize("species", ["proton", "he4", "electron"])
def test_fp64_coefficients_bit_identical(orc, model, species):
    rng = np.random.default_rng(zlib.crc32(f"{model}/{species}".encode()))
    st = _states(300, rng)
    sp = W.SPECIES[species]
    got = _gpu_eval(MODELS[model], sp, 0, st)
    for i in range(st.shape[0]):
        ref = orc.evaluate(MODELS[model], sp, *st[i])
        for j, name in enumerate(cz.DEBUG_EVAL_NAMES):
            a, b = got[i, j], ref[_ORACLE_NAMES[name]]
            assert a == b or (np.isnan(a) and np.isnan(b)), (model, species, i, name, a, b)


@pytest.mark.parametrize("model", list(MODELS))
def test_fp32_coefficients_close(orc, model):
    rng = np.random.default_rng(7)
    st = _states(400, rng)
    sp = W.PROTON
    got = _gpu_eval(MODELS[model], sp, 1, st)
    for i in range(st.shape[0]):
        ref = orc.evaluate(MODELS[model], sp, *st[i])
        scale_v = abs(ref["V"]) + abs(ref["vdr"]) + abs(ref["vdth"]) + abs(ref["vdph"])
        for j, name in enumerate(cz.DEBUG_EVAL_NAMES):
            a, b = got[i, j], ref[_ORACLE_NAMES[name]]
            if name in ("h", "delta_cs") and not MODELS[model]["drift_on"]:
                continue   # the sheet only enters through the drift
            if name in ("vdr", "vdth", "vdph"):
                tol = 2e-3 * scale_v + 1e-6
            elif name in ("Ar", "Ath", "Aph"):
                tol = 2e-4 * (abs(b) + ref["Kpar"] / st[i, 0] ** 2 * 1e-2) + 1e-9
            elif name == "h":
                tol = 2e-3
            elif name == "Krp":
                tol = 1e-4 * ref["Kpar"]
            elif name == "dt":
                tol = 2e-3 * abs(b)
            else:
                tol = 1e-4 * abs(b) + 1e-12
            assert abs(a - b) <= tol, (model, i, name, a, b, st[i])


# ----------------------------------------------------------------- paths --
def test_config0_full_size_fp64(orc):
    job = W.config0()
    g, out, m = gpu_run(job)
    o = orc.job_run(job)
    frac, worst = compare_paths(g, o)
    assert frac >= 0.999 and worst <= 1e-10, (frac, worst)
    assert np.array_equal(g["item"], o["energy"].astype(np.uint32))
    H, J, S = gpu_spectrum(job, out)
    Ho, Jo, So = orc.job_spectrum(job, o)
    assert np.array_equal(H, Ho)
    assert np.allclose(J, Jo, rtol=1e-12, atol=0) and np.allclose(S, So, rtol=1e-10, atol=0)
    m.close()


@pytest.mark.parametrize("model", ["full", "ts_tilt60"])
def test_full_model_fp64_every_path(orc, model):
    T = W.logspace(0.1, 100.0, 10)
    p = dict(MODELS[model])
    job = W.Job(p, W.PROTON, T, [60] * 10, seed=9, bins=W.Bins(0.1, 1000.0, 512))
    g, out, m = gpu_run(job)
    o = orc.job_run(job)
    frac, worst = compare_paths(g, o)
    assert frac >= 0.999 and worst <= 1e-10, (frac, worst)
    H, J, S = gpu_spectrum(job, out)
    Ho, Jo, So = orc.job_spectrum(job, o)
    assert np.array_equal(H, Ho)
    m.close()


def test_config1_full_size_sampled_fp64(orc):
    job = W.config1()
    g, out, m = gpu_run(job)
    assert np.all(g["status"] == cz.PATH_EXIT)
    rng = np.random.default_rng(3)
    sel = np.sort(rng.choice(job.n_particles, size=48, replace=False))
    o = orc.job_run(job, select=sel)
    gs = {k: v[sel] for k, v in g.items()}
    frac, worst = compare_paths(gs, o)
    assert frac == 1.0 and worst <= 1e-10, (frac, worst)
    m.close()


@pytest.mark.parametrize("species", ["he4", "electron"])
def test_species_fp64_paths(orc, species):
    p = W.config3_param_sets()[5]
    job = W.Job(p, W.SPECIES[species], [0.2, 3.0, 40.0], [20, 20, 20], seed=44)
    g, out, m = gpu_run(job)
    o = orc.job_run(job)
    frac, worst = compare_paths(g, o)
    assert frac >= 0.999 and worst <= 1e-10, (frac, worst)
    m.close()


def test_step_limit_state_matches_oracle_trace(orc):
    p = W.params(max_steps=300)
    job = W.Job(p, W.PROTON, [0.5, 5.0], [16, 16], seed=5)
    g, out, m = gpu_run(job)
    assert np.all(g["status"] == cz.PATH_STEP_LIMIT) and np.all(g["steps"] == 300)
    for i in (0, 7, 16, 31):
        tr = orc.trace(p, W.PROTON, job.T_in[i // 16], i, job.seed, 300)
        assert len(tr) == 300
        assert tr[-1, 0] == g["r"][i] and tr[-1, 3] == g["lnP"][i] and tr[-1, 4] == g["s"][i]
    m.close()


def test_ragged_empty_and_host_buffers(orc):
    p = W.config0().params
    job = W.Job(p, W.PROTON, [0.3, 1.0, 2.0, 5.0, 9.0, 20.0], [0, 1, 33, 0, 70, 129], seed=6,
                bins=W.Bins(0.1, 1000.0, 64))
    g, out, m = gpu_run(job)
    o = orc.job_run(job)
    frac, worst = compare_paths(g, o)
    assert frac == 1.0 and worst <= 1e-10
    # the same call writing pinned host buffers gives identical results
    gh, outh, mh = gpu_run(job, host_out=True)
    for k in g:
        assert np.array_equal(g[k], gh[k]), k
    H, J, S = gpu_spectrum(job, out)
    assert np.all(np.isnan(J[[0, 3]])) and np.all(H[[0, 3]] == 0)
    Ho, Jo, So = orc.job_spectrum(job, o)
    assert np.array_equal(H, Ho)
    # no energies at all: a no-op
    empty = W.Job(p, W.PROTON, [], [], seed=1)
    ge, oute, me = gpu_run(empty)
    assert oute.n == 0
    for mm in (m, mh, me):
        mm.close()


def test_invalid_sizes_rejected():
    t = torch()
    job = W.config0(100)
    m = cz.Model(cz.make_params(job.params))
    out = cz.ExitBuffers(99)
    with pytest.raises(cz.CosmicaError) as e:
        cz.cosmica_propagate(m.h, cz.make_species(job.species), job.T_in, job.n_per_energy, 1, out)
    assert e.value.status == cz.ERR_INVALID
    with pytest.raises(cz.CosmicaError):
        cz.cosmica_propagate(m.h, cz.make_species(job.species), [-1.0], [99], 1, out)
    m.close()
