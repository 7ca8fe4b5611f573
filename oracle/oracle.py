"""Python face of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg may import this module.  It compiles and loads ``cosmica_oracle.c`` (plain
C, FP64, -ffp-contract=off) and writes the estimator of Eq. 4 out in numpy.

What each function follows:
  * ``expand``      -- one quasi-particle per (energy bin, sample index) (Sec. IV.A);
  * ``run``         -- the backward Euler-Maruyama loop of Eq. 3 with Eq. 6 (C side);
  * ``histogram``   -- exit rigidities binned on log-spaced bins (Sec. IV.A, binning);
  * ``spectrum``    -- Eq. 4 with L = 0 (Eq. 6) and J = f P^2 (Sec. VI), J the intensity
                       per unit kinetic energy: f is conserved along a path, so
                       f(r0, P0) = <f_LIS(P_exit)> and J(T0) = P0^2 <J_LIS(T_exit) / P_exit^2>.
                       (The energy formulation, Eq. 1 with the loss weight of Eq. 4,
                       gives the same expectation: see ``spectrum_energy_form``.)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cosmica_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libcosmica_oracle.so")

PARAM_FIELDS = (
    "K0", "kperp_r_frac", "kperp_th_frac", "B1AU_nT", "V_slow_kms", "V_fast_kms",
    "lat_fast_deg", "tilt_deg", "polarity", "drift_on", "hcs_on", "R_out", "R_ts",
    "ts_K_factor", "r_in", "dt_max", "dt_fixed", "max_steps", "isotropic",
    "V_const_kms", "eps_adv", "eps_diff", "dt_min", "dlat_deg", "dts_AU",
    "dcs_min_deg", "rot_period_day", "r0", "th0", "ph0", "formulation",
    "n_shells", "shell_blend_AU",
    "squashed", "nose_th", "nose_ph", "ts_tail", "ts_flank", "hp_tail", "hp_flank",
)
MAX_SHELLS = 16
SHELL_ARRAYS = ("shell_K0", "shell_tilt_deg")

EXIT, STEP_LIMIT, NONFINITE = 1, 2, 3

EVAL_NAMES = (
    "P", "beta", "V", "dV_dth", "Gam", "dGam_dr", "dGam_dth",
    "Bmag", "Br", "Bph", "h", "dh_dr", "dh_dth", "dh_dph", "delta_cs",
    "g", "dg_dr", "Kpar",
    "Krr", "Krt", "Krp", "Ktt", "Ktp", "Kpp",
    "dKrr_dr", "dKrp_dr", "dKtt_dth", "dKrr_dth", "dKrp_dth",
    "Ar", "Ath", "Aph",
    "L00", "L10", "L11", "L20", "L21", "L22",
    "Wr", "Wph", "vdr", "vdth", "vdph",
    "dlnP", "Ar_tot", "dt",
    "dg_dth", "dg_dph",
)


class OrcParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in PARAM_FIELDS] + [(n, C.c_double * MAX_SHELLS) for n in SHELL_ARRAYS]


class OrcSpecies(C.Structure):
    _fields_ = [("A", C.c_double), ("Z", C.c_double), ("m0", C.c_double)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
            L.orc_philox_many.argtypes = [C.c_uint64, u32p, u32p, u32p]
            L.orc_normals_many.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, f64p]
            L.orc_eval.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcSpecies),
                                   C.c_double, C.c_double, C.c_double, C.c_double, f64p]
            L.orc_eval_n.restype = C.c_int
            L.orc_run_particles.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcSpecies), C.c_uint64,
                                            u32p, u32p, f64p, u64p, u64p, C.c_void_p,
                                            f64p, f64p, f64p, f64p, f64p, u32p, u8p, f64p, C.c_int]
            L.orc_trace.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcSpecies), C.c_double,
                                    C.c_uint64, C.c_uint64, C.c_uint32, f64p]
            L.orc_trace.restype = C.c_int
            L.orc_max_threads.restype = C.c_int
            L.orc_fn.argtypes = [C.c_int, C.c_uint64, f64p, f64p]
            assert L.orc_eval_n() == len(EVAL_NAMES)
            _lib = L
    return _lib


def _params(p: dict) -> OrcParams:
    o = OrcParams(*[float(p[n]) for n in PARAM_FIELDS])
    for n in SHELL_ARRAYS:
        vals = [float(x) for x in p.get(n, ())]
        getattr(o, n)[:] = (vals + [0.0] * MAX_SHELLS)[:MAX_SHELLS]
    return o


def _species(s: dict) -> OrcSpecies:
    return OrcSpecies(float(s["A"]), float(s["Z"]), float(s["m0"]))


# ------------------------------------------------------------------ RNG --
def philox(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 blocks: ctr is (n, 4) uint32, key two uint32 words."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    lib().orc_philox_many(ctr.shape[0], ctr, k, out)
    return out


def normals(seed: int, pid0: int, n: int, step: int) -> np.ndarray:
    """(n, 3) standard normals of step `step` for particles pid0 .. pid0+n-1."""
    z = np.empty((n, 3), dtype=np.float64)
    lib().orc_normals_many(seed, pid0, n, step, z)
    return z


# ---------------------------------------------------------------- model --
def evaluate(p: dict, species: dict, r: float, th: float, ph: float, lnP: float) -> dict:
    """Every coefficient of one step at (r, th, ph, lnP), by name."""
    out = np.empty(len(EVAL_NAMES), dtype=np.float64)
    lib().orc_eval(C.byref(_params(p)), C.byref(_species(species)), r, th, ph, lnP, out)
    return dict(zip(EVAL_NAMES, out.tolist()))


def rigidity(species: dict, T) -> np.ndarray:
    """P = (A/|Z|) sqrt(T (T + 2 m0)) [GV] for kinetic energy per nucleon T [GeV/n]."""
    T = np.asarray(T, dtype=np.float64)
    return species["A"] / abs(species["Z"]) * np.sqrt(T * (T + 2.0 * species["m0"]))


def kinetic(species: dict, P) -> np.ndarray:
    """T per nucleon from rigidity, in the cancellation-free form p_n^2 / (E_n + m0)."""
    P = np.asarray(P, dtype=np.float64)
    pn = P * abs(species["Z"]) / species["A"]
    return pn * pn / (np.sqrt(pn * pn + species["m0"] ** 2) + species["m0"])


def beta(species: dict, P) -> np.ndarray:
    P = np.asarray(P, dtype=np.float64)
    pn = P * abs(species["Z"]) / species["A"]
    return pn / np.sqrt(pn * pn + species["m0"] ** 2)


# ------------------------------------------------------------ particles --
def expand(n_per_energy, first_pid: int = 0):
    """Work expansion: energy index and particle identity of every quasi-particle."""
    n = np.asarray(n_per_energy, dtype=np.int64)
    e = np.repeat(np.arange(len(n), dtype=np.int64), n)
    pid = first_pid + np.arange(int(n.sum()), dtype=np.uint64)
    return e, pid


def orbit_starts(n_per_energy, positions) -> np.ndarray:
    """Moving detection point (Sec. IV.A): the sample of every energy is divided among the
    orbit's positions (r, th, ph, weight) in proportion to the weights, in position order and
    in contiguous runs: with W_m the sum of the weights before position m and W their total,
    position m takes the particles c_m <= i < c_(m+1), c_m = floor(n W_m / W).
    Returns the start point (r0, th0, ph0) of every particle, in particle order."""
    rows = []
    for n in n_per_energy:
        n = int(n)
        W = 0.0
        for q in positions:
            W += float(q[3])
        cuts, Wm = [], 0.0
        for q in positions:
            cuts.append(math.floor(n * Wm / W))
            Wm += float(q[3])
        cuts.append(n)
        for m, q in enumerate(positions):
            rows += [(float(q[0]), float(q[1]), float(q[2]))] * (cuts[m + 1] - cuts[m])
    return np.array(rows, dtype=np.float64).reshape(-1, 3)


def run(p: dict, species: dict, T_in, n_per_energy, seed: int, select=None, threads: int = 0,
        first_pid: int = 0, positions=None) -> dict:
    """Propagate every quasi-particle of one job (or only the global indices in `select`);
    with `positions`, the start points follow orbit_starts."""
    T_in = np.asarray(T_in, dtype=np.float64)
    e, pid = expand(n_per_energy, first_pid)
    start = None if positions is None else orbit_starts(n_per_energy, positions)
    if select is not None:
        select = np.asarray(select, dtype=np.int64)
        e, pid = e[select], pid[select]
        start = None if start is None else start[select]
    return run_particles([p], [species], np.zeros(len(e), np.uint32), np.zeros(len(e), np.uint32),
                         T_in[e], pid, np.full(len(e), seed, np.uint64), threads, start=start) | {"energy": e}


def run_particles(param_sets, species_list, prm_idx, sp_idx, T, pid, seed, threads: int = 0,
                  start=None) -> dict:
    """start: optional (n, 3) array of per-particle start points (r0, th0, ph0)."""
    n = len(T)
    if start is not None:
        start = np.ascontiguousarray(start, np.float64).reshape(n, 3)
    prm = (OrcParams * max(1, len(param_sets)))(*[_params(p) for p in param_sets])
    spc = (OrcSpecies * max(1, len(species_list)))(*[_species(s) for s in species_list])
    out = {k: np.empty(n, np.float64) for k in ("r", "th", "ph", "lnP", "s")}
    out["steps"] = np.empty(n, np.uint32)
    out["status"] = np.empty(n, np.uint8)
    out["lw"] = np.empty(n, np.float64)
    lib().orc_run_particles(prm, spc, n,
                            np.ascontiguousarray(prm_idx, np.uint32), np.ascontiguousarray(sp_idx, np.uint32),
                            np.ascontiguousarray(T, np.float64), np.ascontiguousarray(pid, np.uint64),
                            np.ascontiguousarray(seed, np.uint64),
                            None if start is None else start.ctypes.data,
                            out["r"], out["th"], out["ph"], out["lnP"], out["s"], out["steps"],
                            out["status"], out["lw"], int(threads))
    return out


def trace(p: dict, species: dict, T_in: float, pid: int, seed: int, nsteps: int) -> np.ndarray:
    out = np.zeros((nsteps, 6), np.float64)
    m = lib().orc_trace(C.byref(_params(p)), C.byref(_species(species)), T_in, pid, seed, nsteps, out)
    return out[:m]


FN_CODES = {"exp": 0, "log": 1, "sin": 2, "cos": 3, "tanh": 4, "atan": 5}


def fn(name: str, x) -> np.ndarray:
    """The oracle's deterministic FP64 elementary function `name` applied element-wise."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty_like(x)
    lib().orc_fn(FN_CODES[name], x.size, x, y)
    return y


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ------------------------------------------------------------ spectrum --
def lis(T) -> np.ndarray:
    """Synthetic local interstellar spectrum per GeV/n: T^-2.7 / (1 + T^-3.7)."""
    T = np.asarray(T, dtype=np.float64)
    return T ** -2.7 / (1.0 + T ** -3.7)


def bin_index(lnP, P_min: float, P_max: float, nbins: int) -> np.ndarray:
    """Bin of log10(P): floor((log10 P - log10 Pmin) / dx); -1 below, nbins above."""
    x_lo = math.log10(P_min)
    dx = (math.log10(P_max) - x_lo) / nbins
    x = np.asarray(lnP, np.float64) / math.log(10.0)
    b = np.floor((x - x_lo) / dx)
    b = np.where(b < 0, -1, np.where(b >= nbins, nbins, b))
    return b.astype(np.int64)


def histogram(run_out: dict, n_energies: int, P_min: float, P_max: float, nbins: int) -> np.ndarray:
    """Per energy: [underflow, bins..., overflow, failed] (failed = step limit or non-finite)."""
    H = np.zeros((n_energies, nbins + 3), np.uint64)
    ok = run_out["status"] == EXIT
    b = bin_index(run_out["lnP"], P_min, P_max, nbins)
    slot = np.where(ok, b + 1, nbins + 2)
    np.add.at(H, (run_out["energy"], slot), 1)
    return H


def bin_centres(P_min: float, P_max: float, nbins: int) -> np.ndarray:
    x_lo = math.log10(P_min)
    dx = (math.log10(P_max) - x_lo) / nbins
    return 10.0 ** (x_lo + (np.arange(nbins) + 0.5) * dx)


def spectrum_from_hist(H: np.ndarray, species: dict, T_in, P_min: float, P_max: float, nbins: int):
    """Binned Eq. 4: J(T0) = P0^2 (1/N) sum_b c_b w_b, w_b = J_LIS(T_b) / P_b^2 at the bin's
    log-centre, sigma = sample std of the summand / sqrt(N).  Under/overflow and failed paths
    are excluded."""
    T_in = np.asarray(T_in, np.float64)
    Pb = bin_centres(P_min, P_max, nbins)
    w = lis(kinetic(species, Pb)) / Pb ** 2
    P0 = rigidity(species, T_in)
    pref = P0 ** 2
    J = np.zeros(len(T_in))
    S = np.zeros(len(T_in))
    for e in range(len(T_in)):
        c = H[e, 1:nbins + 1].astype(np.float64)
        N = c.sum()
        if N == 0:
            J[e], S[e] = math.nan, math.nan
            continue
        mu = (c * w).sum() / N
        var = (c * (w - mu) ** 2).sum() / (N - 1) if N > 1 else 0.0
        J[e] = pref[e] * mu
        S[e] = pref[e] * math.sqrt(var / N)
    return J, S


def spectrum_unbinned(run_out: dict, species: dict, T_in):
    """Unbinned Eq. 4 per energy (each exit rigidity weighted exactly)."""
    T_in = np.asarray(T_in, np.float64)
    ok = run_out["status"] == EXIT
    P = np.exp(run_out["lnP"])
    wt = lis(kinetic(species, P)) / P ** 2
    P0 = rigidity(species, T_in)
    pref = P0 ** 2
    J = np.full(len(T_in), math.nan)
    S = np.full(len(T_in), math.nan)
    for e in range(len(T_in)):
        m = ok & (run_out["energy"] == e)
        if m.sum() == 0:
            continue
        x = wt[m]
        J[e] = pref[e] * x.mean()
        S[e] = pref[e] * (x.std(ddof=1) / math.sqrt(len(x)) if len(x) > 1 else 0.0)
    return J, S


def spectrum_energy_form(run_out: dict, species: dict, T_in):
    """Eq. 4 for the energy formulation (Eq. 1): U = 4 pi J / v is the density per unit
    kinetic energy, so J(T0) / beta0 = <J_LIS(T_exit) exp(-sum L ds) / beta_exit>."""
    T_in = np.asarray(T_in, np.float64)
    ok = run_out["status"] == EXIT
    P = np.exp(run_out["lnP"])
    wt = lis(kinetic(species, P)) * np.exp(run_out["lw"]) / beta(species, P)
    b0 = beta(species, rigidity(species, T_in))
    J = np.full(len(T_in), math.nan)
    S = np.full(len(T_in), math.nan)
    for e in range(len(T_in)):
        m = ok & (run_out["energy"] == e)
        if m.sum() == 0:
            continue
        x = wt[m]
        J[e] = b0[e] * x.mean()
        S[e] = b0[e] * (x.std(ddof=1) / math.sqrt(len(x)) if len(x) > 1 else 0.0)
    return J, S


def job_run(job, select=None, threads: int = 0) -> dict:
    return run(job.params, job.species, job.T_in, job.n_per_energy, job.seed, select, threads)


def job_spectrum(job, out: dict):
    b = job.bins
    H = histogram(out, len(job.T_in), b.P_min, b.P_max, b.n)
    J, S = spectrum_from_hist(H, job.species, job.T_in, b.P_min, b.P_max, b.n)
    return H, J, S
