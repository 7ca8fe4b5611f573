"""Python face of oracle/sde_cartesian.c (test infrastructure only): an
independent Monte Carlo solution of the backward transport SDE stepped in
Cartesian coordinates with finite-difference div K and curl, used by tests/
to pin the oracle's spherical step where the model depends on the longitude
(a tilted current sheet) and no 2-D reduction exists."""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sde_cartesian.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libsde_cartesian.so")

FIELDS = ("K0", "kperp_r", "kperp_th", "B1AU_nT", "V_slow_kms", "V_fast_kms", "lat_fast_deg", "dlat_deg",
          "tilt_deg", "polarity", "drift_on", "hcs_on", "R_out", "R_ts", "ts_K_factor", "dts_AU", "r_in",
          "dt_max", "dt_min", "eps_adv", "eps_diff", "dcs_min_deg", "rot_period_day", "r0", "th0", "ph0",
          "A", "Z", "m0", "max_steps")
# names of the same quantities in the parameter dictionaries of workloads.py
_FROM_PARAMS = {"kperp_r": "kperp_r_frac", "kperp_th": "kperp_th_frac"}


class CartModel(C.Structure):
    _fields_ = [(f, C.c_double) for f in FIELDS]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                        "-o", tmp, SRC, "-lm"], check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
            L.cart_run.argtypes = [C.POINTER(CartModel), C.c_uint64, f64p, u64p, C.c_uint64, f64p, f64p, u32p,
                                   u8p, f64p, C.c_int]
            _lib = L
    return _lib


def model(params: dict, species: dict, step_scale: float = 1.0) -> CartModel:
    """The C record of a parameter set of workloads.py; step_scale multiplies every limit
    of the step rule (eps_adv, eps_diff, dt_max, dt_min)."""
    vals = []
    for f in FIELDS:
        if f in ("A", "Z", "m0"):
            vals.append(float(species[f]))
        elif f in ("dt_max", "dt_min", "eps_adv", "eps_diff"):
            vals.append(float(params[f]) * step_scale)
        else:
            vals.append(float(params[_FROM_PARAMS.get(f, f)]))
    return CartModel(*vals)


def run(params: dict, species: dict, T_in, n_per_energy, seed: int, step_scale: float = 1.0,
        threads: int = 0) -> dict:
    """Paths of every quasi-particle (energy e, index i) with identities 0, 1, ... in order."""
    if params.get("isotropic", 0.0) or params.get("n_shells", 0.0) or params.get("squashed", 0.0):
        raise ValueError("the Cartesian solver covers the full spherical model only")
    if params["kperp_r_frac"] != params["kperp_th_frac"]:
        raise ValueError("needs K_perp,r = K_perp,th (the tensor is then continuous across the polar axis)")
    if params.get("dt_fixed", 0.0) > 0.0 or params.get("formulation", 0.0):
        raise ValueError("adaptive step and momentum form only")
    n = np.asarray(n_per_energy, np.int64)
    e = np.repeat(np.arange(len(n)), n)
    T = np.asarray(T_in, np.float64)[e]
    pid = np.arange(len(T), dtype=np.uint64)
    out = {k: np.empty(len(T), np.float64) for k in ("lnP", "s", "r")}
    out["steps"] = np.empty(len(T), np.uint32)
    out["status"] = np.empty(len(T), np.uint8)
    m = model(params, species, step_scale)
    lib().cart_run(C.byref(m), len(T), np.ascontiguousarray(T), pid, int(seed), out["lnP"], out["s"],
                   out["steps"], out["status"], out["r"], int(threads))
    out["energy"] = e
    return out


def spectrum(run_out: dict, species: dict, T_in):
    """Unbinned Eq. 4 with L = 0: J(T0) = P0^2 <J_LIS(T_exit) / P_exit^2>, sigma its MC error."""
    T_in = np.asarray(T_in, np.float64)
    ok = run_out["status"] == 1
    zoa = abs(species["Z"]) / species["A"]
    P = np.exp(run_out["lnP"])
    pn = P * zoa
    Tex = pn * pn / (np.sqrt(pn * pn + species["m0"] ** 2) + species["m0"])
    w = Tex ** -2.7 / (1.0 + Tex ** -3.7) / P ** 2
    J = np.full(len(T_in), math.nan)
    S = np.full(len(T_in), math.nan)
    for k, T0 in enumerate(T_in):
        m = ok & (run_out["energy"] == k)
        P0 = species["A"] / abs(species["Z"]) * math.sqrt(T0 * (T0 + 2.0 * species["m0"]))
        x = w[m] * P0 * P0
        J[k] = x.mean()
        S[k] = x.std(ddof=1) / math.sqrt(len(x))
    return J, S
