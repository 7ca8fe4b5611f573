"""Seeded synthetic workloads for the COSMICA hot path.

This module only *describes* inputs: parameter sets, species, initial
energies, particle counts, seeds and request arrival times.  It holds none of
the method's arithmetic, so both the FP64 oracle (tests) and the CUDA library
can be fed from it without sharing any computation.

The paper's own workloads (HelMod parameters fitted to AMS-02, the GALPROP
LIS, real isotopes and periods; Sec. II.B, Sec. VII) are not available; the
five workloads below stand in for them with the shapes the paper describes:
one detection point at 1 AU in the ecliptic (Sec. IV.A), independent energy
bins (Sec. IV.A, last paragraph), quasi-particle samples of 10^3..10^5 per
energy (Sec. VII), and protons / helium / electrons as species.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Tuple

import numpy as np

# Species: mass number A, signed charge Z, rest mass per nucleon m0 [GeV].
PROTON = {"A": 1, "Z": 1, "m0": 0.93827208816}
HELIUM4 = {"A": 4, "Z": 2, "m0": 3.7273794 / 4.0}
ELECTRON = {"A": 1, "Z": -1, "m0": 0.51099895e-3}
SPECIES = {"proton": PROTON, "he4": HELIUM4, "electron": ELECTRON}

# Field order of the parameter record (the C structs on both sides use it).
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
SHELL_ARRAYS = ("shell_K0", "shell_tilt_deg")   # per-shell tables (lists of up to 16 values)

DEFAULT_PARAMS: Dict[str, float] = {
    "K0": 11.5,             # AU^2/day
    "kperp_r_frac": 0.02,
    "kperp_th_frac": 0.02,
    "B1AU_nT": 5.0,
    "V_slow_kms": 400.0,
    "V_fast_kms": 760.0,
    "lat_fast_deg": 30.0,
    "tilt_deg": 20.0,
    "polarity": 1.0,
    "drift_on": 1.0,
    "hcs_on": 1.0,
    "R_out": 100.0,         # AU
    "R_ts": 0.0,            # AU, 0 = no termination shock
    "ts_K_factor": 0.5,
    "r_in": 0.1,            # AU
    "dt_max": 0.1,          # day
    "dt_fixed": 0.0,        # day, 0 = adaptive
    "max_steps": 1.0e8,
    "isotropic": 0.0,
    "V_const_kms": 400.0,
    "eps_adv": 0.01,
    "eps_diff": 0.01,
    "dt_min": 1.0e-4,       # day
    "dlat_deg": 2.0,
    "dts_AU": 1.0,
    "dcs_min_deg": 1.0,
    "rot_period_day": 25.38,
    "r0": 1.0,
    "th0": math.pi / 2.0,
    "ph0": 0.0,
    "formulation": 0.0,     # 0: momentum form (Eq. 5-6); 1: energy form with loss weight (Eq. 1, Eq. 4)
    "n_shells": 0.0,        # radial shells of the inner heliosphere (0: one region)
    "shell_blend_AU": 0.5,  # half-width of the blend across each interior shell edge
    "squashed": 0.0,        # 1: shock and outer boundary are spheroids squashed toward the nose
    "nose_th": math.pi / 2.0,   # nose direction (colatitude, longitude) [rad]
    "nose_ph": 0.0,
    "ts_tail": 1.0,         # shock: tail distance / nose distance (R_ts)
    "ts_flank": 1.0,        # shock: flank semi-axis / nose distance
    "hp_tail": 1.0,         # outer boundary: the same ratios (R_out at the nose)
    "hp_flank": 1.0,
    "shell_K0": (),         # K0 of each shell [AU^2/day], innermost first
    "shell_tilt_deg": (),   # current-sheet tilt of each shell [deg]
}


def params(**overrides) -> Dict[str, float]:
    p = dict(DEFAULT_PARAMS)
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = tuple(float(x) for x in v) if k in SHELL_ARRAYS else float(v)
    return p


@dataclass
class Bins:
    """Log-spaced rigidity bins for the exit histogram."""
    P_min: float = 0.1      # GV
    P_max: float = 1000.0   # GV
    n: int = 512


@dataclass
class Job:
    """One spectrum: one parameter set, one species, several energies."""
    params: Dict[str, float]
    species: Dict[str, float]
    T_in: List[float]
    n_per_energy: List[int]
    seed: int
    bins: Bins = field(default_factory=Bins)
    name: str = ""
    mixed: bool = False     # mixed precision (FP32 evaluation, compensated accumulation)

    @property
    def n_particles(self) -> int:
        return int(sum(self.n_per_energy))


# Particle identities of a rank's replica start at rank * PID_STRIDE (weak scaling).
PID_STRIDE = 1 << 40


def items_of(jobs, rank: int = 0):
    """Work items (param_idx, species_idx, T, n, first_pid, seed) of all jobs, with
    de-duplicated parameter sets and species.  rank > 0 gives the replica of that
    rank (identities and seeds offset); the partition uses rank 0's list."""
    params, pkeys, species, skeys, items = [], {}, [], {}, []
    pid = 0
    base = rank * PID_STRIDE
    for j in jobs:
        pk = tuple(sorted(j.params.items()))
        if pk not in pkeys:
            pkeys[pk] = len(params)
            params.append(j.params)
        sk = tuple(sorted(j.species.items()))
        if sk not in skeys:
            skeys[sk] = len(species)
            species.append(j.species)
        for T, n in zip(j.T_in, j.n_per_energy):
            items.append((pkeys[pk], skeys[sk], T, n, base + pid, j.seed + 7919 * rank))
            pid += n
    if pid >= PID_STRIDE:
        raise ValueError("workload exceeds the per-rank particle-identity range")
    return params, species, items


def logspace(lo: float, hi: float, n: int) -> List[float]:
    return [float(x) for x in np.logspace(math.log10(lo), math.log10(hi), n)]


# ---------------------------------------------------------------- configs --
def config0(n: int = 10_000) -> Job:
    """Isotropic K = K0 beta P, uniform 400 km/s wind, 100 AU, dt = 0.1 day, 1 GeV protons."""
    p = params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, V_const_kms=400.0,
               dt_fixed=0.1, R_out=100.0)
    return Job(p, PROTON, [1.0], [n], seed=1, bins=Bins(0.1, 1000.0, 64), name="c0")


def config1(n_per: int = 5_000, n_e: int = 10) -> Job:
    """Full heliospheric model in FP64: Parker field, two-speed wind, drifts, wavy sheet, tilt 20, qA > 0."""
    return Job(params(), PROTON, logspace(0.1, 100.0, n_e), [n_per] * n_e, seed=1,
               bins=Bins(0.1, 1000.0, 512), name="c1")


def config2(n_per: int = 20_000, n_e: int = 30) -> Job:
    """Config 1 in mixed precision, 30 energies x 20 000."""
    j = config1(n_per, n_e)
    j.name, j.mixed = "c2", True
    return j


def polar_orbit(n_pos: int = 12, a_AU: float = 3.35, e: float = 0.6,
                incl_deg: float = 80.0) -> List[Tuple[float, float, float, float]]:
    """A synthetic out-of-ecliptic orbit for the moving detection point (Sec. IV.A): a Kepler
    ellipse of semi-major axis a_AU and eccentricity e (perihelion 1.34 AU, aphelion 5.36 AU by
    default) inclined incl_deg to the ecliptic, with its perihelion on the line of nodes, so
    that the latitude sweeps fastest near the Sun.  Sampled at n_pos equal steps of mean
    anomaly, i.e. of time: (r [AU], theta [rad], phi [rad], weight 1) per position."""
    out = []
    inc = math.radians(incl_deg)
    for k in range(n_pos):
        M = 2.0 * math.pi * (k + 0.5) / n_pos
        E = M + e * math.sin(M)
        for _ in range(60):                       # Kepler's equation E - e sin E = M
            E -= (E - e * math.sin(E) - M) / (1.0 - e * math.cos(E))
        r = a_AU * (1.0 - e * math.cos(E))
        nu = 2.0 * math.atan2(math.sqrt(1.0 + e) * math.sin(E / 2.0), math.sqrt(1.0 - e) * math.cos(E / 2.0))
        x, y, z = r * math.cos(nu), r * math.sin(nu) * math.cos(inc), r * math.sin(nu) * math.sin(inc)
        out.append((r, math.acos(z / r), math.atan2(y, x) % (2.0 * math.pi), 1.0))
    return out


def config3_param_sets(seed: int = 20250210, n_sets: int = 64) -> List[Dict[str, float]]:
    """64 heliospheres: K0 ~ U[5,30], tilt ~ U[5,75] deg, polarity +-1, V_slow ~ U[300,500] km/s,
    termination shock at 85 AU with x0.5 diffusion beyond, heliopause boundary at 122 AU."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_sets):
        out.append(params(
            K0=rng.uniform(5.0, 30.0),
            tilt_deg=rng.uniform(5.0, 75.0),
            polarity=1.0 if rng.integers(0, 2) == 1 else -1.0,
            V_slow_kms=rng.uniform(300.0, 500.0),
            R_ts=85.0, ts_K_factor=0.5, R_out=122.0))
    return out


# Nose-squashed heliosphere (Sec. II.B): shock 85 AU at the nose, 1.35x at the tail, 1.15x
# on the flanks; outer boundary 122 AU at the nose, 1.6x / 1.25x; nose 5 deg south of the
# ecliptic.  A synthetic shape of the right proportions (HelMod's fitted surfaces are not
# available).
SQUASHED = {"squashed": 1.0, "nose_th": math.pi / 2.0 + math.radians(5.0), "nose_ph": math.radians(255.0),
            "ts_tail": 1.35, "ts_flank": 1.15, "hp_tail": 1.6, "hp_flank": 1.25}


def config3(seed: int = 20250210, n_sets: int = 64, n_e: int = 30,
            n_lo: int = 1_000, n_hi: int = 50_000, scale: float = 1.0, geometry=None) -> List[Job]:
    """Batched workload: 64 parameter sets x {proton, He-4, electron} x 30 energies,
    uneven log-uniform counts in [n_lo, n_hi] (scaled by `scale`); `geometry` overrides
    the boundary shape (e.g. SQUASHED)."""
    sets = config3_param_sets(seed, n_sets)
    if geometry:
        sets = [dict(p, **{k: float(v) for k, v in geometry.items()}) for p in sets]
    rng = np.random.default_rng(seed + 1)
    T = logspace(0.1, 100.0, n_e)
    jobs = []
    for i, p in enumerate(sets):
        for sname in ("proton", "he4", "electron"):
            counts = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_e))
            counts = [max(1, int(round(c * scale))) for c in counts]
            jobs.append(Job(p, SPECIES[sname], T, counts,
                            seed=seed * 1000 + len(jobs), bins=Bins(0.1, 1000.0, 512),
                            name=f"c3/{i}/{sname}", mixed=True))
    return jobs


# ------------------------------------------------ time-dependent shells --
CARRINGTON_DAYS = 27.26     # synodic rotation period (Sec. II.B)
CYCLE_ROTATIONS = 147.3     # ~11-year solar cycle in Carrington rotations


def solar_cycle_series(seed: int = 20250212, n_rot: int = 200) -> Dict[str, List[float]]:
    """Synthetic solar activity per Carrington rotation (the paper's HelMod tables are
    not available): activity a = sin^2(pi c / 147.3); current-sheet tilt 8 + 62 a deg and
    diffusion normalisation K0 = 30 - 22 a AU^2/day, each with seeded noise and clipped to
    config 3's ranges ([5, 75] deg, [5, 30] AU^2/day)."""
    rng = np.random.default_rng(seed)
    c = np.arange(n_rot)
    a = np.sin(np.pi * c / CYCLE_ROTATIONS) ** 2
    tilt = np.clip(8.0 + 62.0 * a + rng.normal(0.0, 3.0, n_rot), 5.0, 75.0)
    K0 = np.clip(30.0 - 22.0 * a + rng.normal(0.0, 1.0, n_rot), 5.0, 30.0)
    return {"K0": [float(x) for x in K0], "tilt_deg": [float(x) for x in tilt]}


def shell_params(series, rotation: int, n_shells: int = 15, **overrides) -> Dict[str, float]:
    """Heliosphere observed at Carrington rotation `rotation`: shell k (innermost k = 0)
    holds the conditions of rotation `rotation - k`, whose wind fills it (Sec. II.B)."""
    if rotation - (n_shells - 1) < 0:
        raise ValueError("the series must reach n_shells - 1 rotations back")
    K0 = [series["K0"][rotation - k] for k in range(n_shells)]
    tilt = [series["tilt_deg"][rotation - k] for k in range(n_shells)]
    base = dict(R_ts=85.0, ts_K_factor=0.5, R_out=122.0, K0=K0[0], tilt_deg=tilt[0],
                n_shells=n_shells, shell_K0=K0, shell_tilt_deg=tilt)
    base.update(overrides)
    return params(**base)


def config_shells(seed: int = 20250212, first_rotation: int = 40, n_obs: int = 13, n_e: int = 30,
                  n_lo: int = 1_000, n_hi: int = 50_000, scale: float = 1.0) -> List[Job]:
    """Time-dependent batch: one observation per Carrington rotation over a year (13
    rotations), each a heliosphere of 15 radial shells from the synthetic solar-cycle
    series; protons and He-4, 30 energies, log-uniform counts in [n_lo, n_hi]."""
    ser = solar_cycle_series(seed)
    rng = np.random.default_rng(seed + 1)
    T = logspace(0.1, 100.0, n_e)
    jobs = []
    for i in range(n_obs):
        p = shell_params(ser, first_rotation + i)
        for sname in ("proton", "he4"):
            counts = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_e))
            counts = [max(1, int(round(c * scale))) for c in counts]
            jobs.append(Job(p, SPECIES[sname], T, counts, seed=seed * 1000 + len(jobs),
                            bins=Bins(0.1, 1000.0, 512), name=f"shells/{i}/{sname}", mixed=True))
    return jobs


@dataclass
class Request:
    t_arrival: float        # seconds from the start of the stream
    job: Job


def config4(seed: int = 20250211, n_requests: int = 200, rate_hz: float = 200.0,
            n_lo: int = 2_000, n_hi: int = 100_000, scale: float = 1.0) -> List[Request]:
    """Serving stream: Poisson arrivals, each request one parameter set from config 3's
    ranges, one species, 4-30 energies with log-uniform counts in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    names = ("proton", "he4", "electron")
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        p = params(K0=rng.uniform(5.0, 30.0), tilt_deg=rng.uniform(5.0, 75.0),
                   polarity=1.0 if rng.integers(0, 2) == 1 else -1.0,
                   V_slow_kms=rng.uniform(300.0, 500.0),
                   R_ts=85.0, ts_K_factor=0.5, R_out=122.0)
        sp = SPECIES[names[int(rng.integers(0, 3))]]
        n_e = int(rng.integers(4, 31))
        T = sorted(float(x) for x in np.exp(rng.uniform(math.log(0.1), math.log(100.0), n_e)))
        counts = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_e))
        counts = [max(1, int(round(c * scale))) for c in counts]
        out.append(Request(t, Job(p, sp, T, counts, seed=seed * 1000 + i,
                                  bins=Bins(0.1, 1000.0, 512), name=f"c4/{i}", mixed=True)))
    return out
