"""ctypes binding of libcosmica (include/cosmica.h, include/cosmica_debug.h).

Argument marshalling only: every step of the propagation path runs in the
library's CUDA kernels.  PyTorch provides device memory and streams; the
functions accept torch tensors (their data pointers are passed) and the
current torch CUDA stream by default.  If the compiled library is missing or
cannot be loaded, every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from typing import Optional, Sequence

from . import _build

# ------------------------------------------------------------ ABI mirror --
ABI_VERSION = 1
PREC_FP64, PREC_MIXED, PREC_MIXED_F64ACC = 0, 1, 2
PATH_RUNNING, PATH_EXIT, PATH_STEP_LIMIT, PATH_NONFINITE = 0, 1, 2, 3
OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY = range(6)
DEBUG_EVAL_N = 21
DEBUG_EVAL_NAMES = ("V", "Gam", "Kpar", "Krr", "Ktt", "Kpp", "Krp", "Ar", "Ath", "Aph", "L00", "L11",
                    "L20", "L22", "h", "delta_cs", "vdr", "vdth", "vdph", "dlnP", "dt")


class cosmica_params(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("version", C.c_uint32),
        ("K0", C.c_double), ("kperp_r_frac", C.c_double), ("kperp_th_frac", C.c_double),
        ("B1AU_nT", C.c_double), ("V_slow_kms", C.c_double), ("V_fast_kms", C.c_double),
        ("lat_fast_deg", C.c_double), ("tilt_deg", C.c_double),
        ("polarity", C.c_int32), ("drift_on", C.c_int32), ("hcs_on", C.c_int32), ("isotropic", C.c_int32),
        ("R_out_AU", C.c_double), ("R_ts_AU", C.c_double), ("ts_K_factor", C.c_double), ("r_in_AU", C.c_double),
        ("dt_max_day", C.c_double), ("dt_fixed_day", C.c_double), ("dt_min_day", C.c_double),
        ("eps_adv", C.c_double), ("eps_diff", C.c_double), ("V_const_kms", C.c_double),
        ("dlat_deg", C.c_double), ("dts_AU", C.c_double), ("dcs_min_deg", C.c_double),
        ("rot_period_day", C.c_double), ("r0_AU", C.c_double), ("th0_rad", C.c_double), ("ph0_rad", C.c_double),
        ("max_steps", C.c_uint32), ("precision", C.c_int32), ("formulation", C.c_int32),
        ("reserved0", C.c_int32),
        ("n_shells", C.c_uint32), ("reserved1", C.c_uint32), ("shell_blend_AU", C.c_double),
        ("shell_K0", C.c_double * 16), ("shell_tilt_deg", C.c_double * 16),
        ("squashed", C.c_int32), ("reserved2", C.c_int32), ("nose_th_rad", C.c_double), ("nose_ph_rad", C.c_double),
        ("ts_tail_ratio", C.c_double), ("ts_flank_ratio", C.c_double), ("hp_tail_ratio", C.c_double),
        ("hp_flank_ratio", C.c_double),
    ]


class cosmica_species(C.Structure):
    _fields_ = [("A", C.c_int32), ("Z", C.c_int32), ("m0_GeV", C.c_double)]


class cosmica_exit_states(C.Structure):
    _fields_ = [("r", C.c_void_p), ("th", C.c_void_p), ("ph", C.c_void_p), ("lnP", C.c_void_p),
                ("s", C.c_void_p), ("steps", C.c_void_p), ("status", C.c_void_p), ("item", C.c_void_p),
                ("n", C.c_uint64), ("lw", C.c_void_p)]


class cosmica_lis(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_uint32), ("lnT", C.c_void_p), ("lnJ", C.c_void_p)]


class cosmica_bins(C.Structure):
    _fields_ = [("P_min_GV", C.c_double), ("P_max_GV", C.c_double), ("nbins", C.c_uint32)]


class cosmica_work_item(C.Structure):
    _fields_ = [("param_idx", C.c_uint32), ("species_idx", C.c_uint32), ("T_GeVn", C.c_double),
                ("n", C.c_uint32), ("exit_item_plus1", C.c_uint32), ("first_pid", C.c_uint64),
                ("seed", C.c_uint64),
                ("r0_AU", C.c_double), ("th0_rad", C.c_double), ("ph0_rad", C.c_double)]


class cosmica_position(C.Structure):
    _fields_ = [("r_AU", C.c_double), ("th_rad", C.c_double), ("ph_rad", C.c_double), ("weight", C.c_double)]


class cosmica_tuning(C.Structure):
    _fields_ = [("block", C.c_uint32), ("blocks_per_sm", C.c_uint32), ("compact_period", C.c_uint32),
                ("use_graph", C.c_uint32), ("queue_order", C.c_uint32)]


class cosmica_request(C.Structure):
    _fields_ = [("params", cosmica_params), ("species", cosmica_species), ("T_GeVn", C.c_void_p),
                ("n_per_energy", C.c_void_p), ("n_energies", C.c_uint32), ("seed", C.c_uint64),
                ("bins", cosmica_bins)]


class cosmica_result(C.Structure):
    _fields_ = [("J", C.c_void_p), ("sigma", C.c_void_p), ("hist", C.c_void_p), ("steps", C.c_uint64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class cosmica_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("rejected", C.c_uint64), ("quanta", C.c_uint64), ("steps", C.c_uint64),
                ("in_flight_particles", C.c_uint64), ("arena_capacity", C.c_uint64), ("arena_used", C.c_uint64),
                ("busy_seconds", C.c_double)]


class CosmicaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cosmica status {status}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()
P = C.c_void_p


def lib():
    """Load libcosmica.so (compiling it with nvcc first if the sources changed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            s = C.c_int
            L.cosmica_params_default.argtypes = [C.POINTER(cosmica_params)]
            L.cosmica_model_create.argtypes = [C.POINTER(cosmica_params), C.POINTER(P)]
            L.cosmica_model_destroy.argtypes = [P]
            L.cosmica_propagate.argtypes = [P, C.POINTER(cosmica_species), C.POINTER(C.c_double), C.c_uint32,
                                            C.POINTER(C.c_uint32), C.c_uint64, C.POINTER(cosmica_exit_states), P]
            L.cosmica_spectrum.argtypes = [C.POINTER(cosmica_exit_states), C.POINTER(cosmica_species),
                                           C.POINTER(C.c_double), C.c_uint32, C.POINTER(cosmica_lis),
                                           C.POINTER(cosmica_bins), P, P, P, P]
            L.cosmica_spectrum_unbinned.argtypes = [C.POINTER(cosmica_exit_states), C.POINTER(cosmica_species),
                                                    C.POINTER(C.c_double), C.c_uint32, C.POINTER(C.c_uint32),
                                                    C.c_int32, C.POINTER(cosmica_lis), P, P, P]
            L.cosmica_spectrum_unbinned.restype = C.c_int
            L.cosmica_batch_create.argtypes = [C.POINTER(cosmica_params), C.c_uint32, C.POINTER(cosmica_species),
                                               C.c_uint32, C.POINTER(P)]
            L.cosmica_batch_destroy.argtypes = [P]
            L.cosmica_batch_run.argtypes = [P, C.POINTER(cosmica_work_item), C.c_uint32, C.POINTER(cosmica_tuning),
                                            C.POINTER(cosmica_exit_states), P, P]
            L.cosmica_batch_spectrum.argtypes = [P, C.POINTER(cosmica_work_item), C.c_uint32,
                                                 C.POINTER(cosmica_exit_states), C.POINTER(cosmica_lis),
                                                 C.POINTER(cosmica_bins), P, P, P, P]
            L.cosmica_batch_spectrum_hist.argtypes = [P, C.POINTER(cosmica_work_item), C.c_uint32,
                                                      C.POINTER(cosmica_lis), C.POINTER(cosmica_bins), P, P, P, P]
            L.cosmica_autotune.argtypes = [P, C.POINTER(cosmica_work_item), C.c_uint32, C.POINTER(cosmica_tuning),
                                           C.POINTER(C.c_double)]
            L.cosmica_propagate_noalloc.argtypes = [C.POINTER(cosmica_params), C.POINTER(cosmica_species),
                                                    C.POINTER(C.c_double), C.c_uint32, C.POINTER(C.c_uint32),
                                                    C.c_uint64, C.POINTER(cosmica_exit_states), P]
            L.cosmica_propagate_noalloc.restype = C.c_int
            L.cosmica_propagate_orbit.argtypes = [P, C.POINTER(cosmica_species), C.POINTER(C.c_double), C.c_uint32,
                                                  C.POINTER(C.c_uint32), C.POINTER(cosmica_position), C.c_uint32,
                                                  C.c_uint64, C.POINTER(cosmica_exit_states), P]
            L.cosmica_propagate_orbit.restype = C.c_int
            L.cosmica_server_create.argtypes = [C.c_size_t, C.c_int32, C.c_uint32, C.POINTER(P)]
            L.cosmica_server_submit.argtypes = [P, C.POINTER(cosmica_request), C.POINTER(C.c_uint64)]
            L.cosmica_server_poll.argtypes = [P, C.c_uint64, C.POINTER(cosmica_result)]
            L.cosmica_server_wait.argtypes = [P, C.c_uint64, C.c_uint32, C.POINTER(cosmica_result)]
            L.cosmica_server_stats_get.argtypes = [P, C.POINTER(cosmica_server_stats)]
            L.cosmica_server_destroy.argtypes = [P]
            for name in ("cosmica_server_create", "cosmica_server_submit", "cosmica_server_poll",
                         "cosmica_server_wait", "cosmica_server_stats_get"):
                getattr(L, name).restype = C.c_int
            L.cosmica_last_error.restype = C.c_char_p
            L.cosmica_launch_count.restype = C.c_uint64
            L.cosmica_debug_philox.argtypes = [C.c_uint32, P, C.c_uint32, C.c_uint32, P, P]
            L.cosmica_debug_curand_philox.argtypes = [C.c_uint32, C.c_uint64, P, P, P, P]
            L.cosmica_debug_normals64.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, P, P]
            L.cosmica_debug_normals32.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, P, P, P]
            L.cosmica_debug_fn64.argtypes = [C.c_int32, C.c_uint32, P, P, P]
            L.cosmica_debug_eval.argtypes = [P, C.POINTER(cosmica_species), C.c_int32, C.c_uint32, P, P, P]
            for name in ("cosmica_model_create", "cosmica_propagate", "cosmica_spectrum", "cosmica_batch_create",
                         "cosmica_batch_run", "cosmica_batch_spectrum", "cosmica_batch_spectrum_hist", "cosmica_autotune", "cosmica_debug_philox",
                         "cosmica_debug_curand_philox", "cosmica_debug_normals64", "cosmica_debug_normals32", "cosmica_debug_fn64",
                         "cosmica_debug_eval"):
                getattr(L, name).restype = s
            _lib = L
    return _lib


def _check(st: int):
    if st != OK:
        raise CosmicaError(st, lib().cosmica_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------- marshalling --
_PARAM_MAP = {
    "K0": "K0", "kperp_r_frac": "kperp_r_frac", "kperp_th_frac": "kperp_th_frac", "B1AU_nT": "B1AU_nT",
    "V_slow_kms": "V_slow_kms", "V_fast_kms": "V_fast_kms", "lat_fast_deg": "lat_fast_deg",
    "tilt_deg": "tilt_deg", "polarity": "polarity", "drift_on": "drift_on", "hcs_on": "hcs_on",
    "isotropic": "isotropic", "R_out": "R_out_AU", "R_ts": "R_ts_AU", "ts_K_factor": "ts_K_factor",
    "r_in": "r_in_AU", "dt_max": "dt_max_day", "dt_fixed": "dt_fixed_day", "dt_min": "dt_min_day",
    "eps_adv": "eps_adv", "eps_diff": "eps_diff", "V_const_kms": "V_const_kms", "dlat_deg": "dlat_deg",
    "dts_AU": "dts_AU", "dcs_min_deg": "dcs_min_deg", "rot_period_day": "rot_period_day",
    "r0": "r0_AU", "th0": "th0_rad", "ph0": "ph0_rad", "max_steps": "max_steps",
    "formulation": "formulation", "n_shells": "n_shells", "shell_blend_AU": "shell_blend_AU",
    "shell_K0": "shell_K0", "shell_tilt_deg": "shell_tilt_deg",
    "squashed": "squashed", "nose_th": "nose_th_rad", "nose_ph": "nose_ph_rad", "ts_tail": "ts_tail_ratio",
    "ts_flank": "ts_flank_ratio", "hp_tail": "hp_tail_ratio", "hp_flank": "hp_flank_ratio",
}
_INT_FIELDS = {"polarity", "drift_on", "hcs_on", "isotropic", "max_steps", "formulation", "n_shells", "squashed"}
_ARRAY_FIELDS = {"shell_K0", "shell_tilt_deg"}


def make_params(d: dict, precision: int = PREC_FP64) -> cosmica_params:
    p = cosmica_params()
    lib().cosmica_params_default(C.byref(p))
    for k, v in d.items():
        f = _PARAM_MAP[k]
        if f in _ARRAY_FIELDS:
            vals = [float(x) for x in v]
            getattr(p, f)[:] = (vals + [0.0] * 16)[:16]
        else:
            setattr(p, f, int(round(v)) if f in _INT_FIELDS else float(v))
    p.precision = int(precision)
    return p


def make_species(d: dict) -> cosmica_species:
    return cosmica_species(int(d["A"]), int(d["Z"]), float(d["m0"]))


def make_bins(P_min: float, P_max: float, n: int) -> cosmica_bins:
    return cosmica_bins(float(P_min), float(P_max), int(n))


class ExitBuffers:
    """Exit-state SoA (torch tensors) and its ctypes view."""

    def __init__(self, n: int, device="cuda", pin_memory: bool = False, with_lw: bool = False):
        import torch
        kw = dict(device=device)
        if device == "cpu" and pin_memory:
            kw = dict(device="cpu", pin_memory=True)
        self.n = int(n)
        self.r = torch.empty(self.n, dtype=torch.float64, **kw)
        self.th = torch.empty(self.n, dtype=torch.float64, **kw)
        self.ph = torch.empty(self.n, dtype=torch.float64, **kw)
        self.lnP = torch.empty(self.n, dtype=torch.float64, **kw)
        self.s = torch.empty(self.n, dtype=torch.float64, **kw)
        self.steps = torch.empty(self.n, dtype=torch.int32, **kw)    # uint32 bits
        self.status = torch.empty(self.n, dtype=torch.uint8, **kw)
        self.item = torch.empty(self.n, dtype=torch.int32, **kw)     # uint32 bits
        self.lw = torch.empty(self.n, dtype=torch.float64, **kw) if with_lw else None
        self.c = cosmica_exit_states(*[_ptr(t) for t in (self.r, self.th, self.ph, self.lnP, self.s,
                                                         self.steps, self.status, self.item)], self.n,
                                     _ptr(self.lw))

    def numpy(self) -> dict:
        import numpy as np
        out = {k: getattr(self, k).cpu().numpy() for k in ("r", "th", "ph", "lnP", "s", "status")}
        out["steps"] = self.steps.cpu().numpy().view(np.uint32)
        out["item"] = self.item.cpu().numpy().view(np.uint32)
        if self.lw is not None:
            out["lw"] = self.lw.cpu().numpy()
        return out

    @property
    def nbytes(self) -> int:
        """Bytes of the exit records: r, th, ph, lnP, s (f64), steps, item (u32), status (u8), lw (f64)."""
        return self.n * (5 * 8 + 4 + 1 + 4 + (8 if self.lw is not None else 0))


# --------------------------------------------------------------- model API --
class Model:
    """Owner of a cosmica_model handle."""

    def __init__(self, params: cosmica_params):
        self.h = cosmica_model_create(params)
        self.precision = params.precision

    def close(self):
        if self.h:
            cosmica_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cosmica_model_create(params: cosmica_params) -> int:
    h = P()
    _check(lib().cosmica_model_create(C.byref(params), C.byref(h)))
    return h.value


def cosmica_model_destroy(h: int) -> None:
    lib().cosmica_model_destroy(h)


def cosmica_propagate(model: int, species: cosmica_species, T_in: Sequence[float], n_per_energy: Sequence[int],
                      seed: int, out: ExitBuffers, stream=None) -> None:
    n = len(T_in)
    T = (C.c_double * max(1, n))(*[float(t) for t in T_in])
    N = (C.c_uint32 * max(1, n))(*[int(x) for x in n_per_energy])
    _check(lib().cosmica_propagate(model, C.byref(species), T, n, N, int(seed), C.byref(out.c), _stream(stream)))


def cosmica_propagate_orbit(model: int, species: cosmica_species, T_in: Sequence[float],
                            n_per_energy: Sequence[int], positions, seed: int, out: ExitBuffers,
                            stream=None) -> None:
    """positions: iterable of (r_AU, th_rad, ph_rad, weight)."""
    n = len(T_in)
    T = (C.c_double * max(1, n))(*[float(t) for t in T_in])
    N = (C.c_uint32 * max(1, n))(*[int(x) for x in n_per_energy])
    pos = list(positions)
    arr = (cosmica_position * max(1, len(pos)))(*[cosmica_position(*map(float, q)) for q in pos])
    _check(lib().cosmica_propagate_orbit(model, C.byref(species), T, n, N, arr, len(pos), int(seed),
                                         C.byref(out.c), _stream(stream)))


def cosmica_propagate_noalloc(params: cosmica_params, species: cosmica_species, T_in: Sequence[float],
                              n_per_energy: Sequence[int], seed: int, out: ExitBuffers, stream=None) -> None:
    """Allocation-free propagation: scratch in a fixed static device array (see cosmica.h)."""
    n = len(T_in)
    T = (C.c_double * max(1, n))(*[float(t) for t in T_in])
    N = (C.c_uint32 * max(1, n))(*[int(x) for x in n_per_energy])
    _check(lib().cosmica_propagate_noalloc(C.byref(params), C.byref(species), T, n, N, int(seed), C.byref(out.c),
                                           _stream(stream)))


def cosmica_spectrum(exit: ExitBuffers, species: cosmica_species, T_in: Sequence[float], bins: cosmica_bins,
                     J, sigma, hist, lis: Optional[cosmica_lis] = None, stream=None) -> None:
    n = len(T_in)
    T = (C.c_double * max(1, n))(*[float(t) for t in T_in])
    lp = C.byref(lis) if lis is not None else None
    _check(lib().cosmica_spectrum(C.byref(exit.c), C.byref(species), T, n, lp, C.byref(bins), _ptr(J),
                                  _ptr(sigma), _ptr(hist), _stream(stream)))


def cosmica_spectrum_unbinned(exit: ExitBuffers, species: cosmica_species, T_in: Sequence[float],
                              n_per_energy: Sequence[int], formulation: int, J, sigma,
                              lis: Optional[cosmica_lis] = None, stream=None) -> None:
    n = len(T_in)
    T = (C.c_double * max(1, n))(*[float(t) for t in T_in])
    N = (C.c_uint32 * max(1, n))(*[int(x) for x in n_per_energy])
    lp = C.byref(lis) if lis is not None else None
    _check(lib().cosmica_spectrum_unbinned(C.byref(exit.c), C.byref(species), T, n, N, int(formulation), lp,
                                           _ptr(J), _ptr(sigma), _stream(stream)))


# --------------------------------------------------------------- batch API --
def make_items(items, exit_items=None) -> "C.Array":
    """items: iterable of (param_idx, species_idx, T, n, first_pid, seed[, (r0, th0, ph0)]);
    without the start position the parameter set's is used.  exit_items: optional
    item number each item's exit records carry (default: its index in `items`)."""
    items = list(items)
    arr = (cosmica_work_item * max(1, len(items)))()
    for i, it in enumerate(items):
        pi, si, T, n, fp, sd = it[:6]
        r0, th0, ph0 = it[6] if len(it) > 6 and it[6] is not None else (0.0, 0.0, 0.0)
        tag = 0 if exit_items is None else int(exit_items[i]) + 1
        arr[i] = cosmica_work_item(int(pi), int(si), float(T), int(n), tag, int(fp), int(sd),
                                   float(r0), float(th0), float(ph0))
    return arr


def cosmica_batch_create(params: Sequence[cosmica_params], species: Sequence[cosmica_species]) -> int:
    pa = (cosmica_params * len(params))(*params)
    sa = (cosmica_species * len(species))(*species)
    h = P()
    _check(lib().cosmica_batch_create(pa, len(params), sa, len(species), C.byref(h)))
    return h.value


def cosmica_batch_destroy(h: int) -> None:
    lib().cosmica_batch_destroy(h)


def cosmica_batch_run(batch: int, items, n_items: int, out: ExitBuffers, tuning: Optional[cosmica_tuning] = None,
                      steps_out=None, stream=None) -> None:
    tp = C.byref(tuning) if tuning is not None else None
    _check(lib().cosmica_batch_run(batch, items, n_items, tp, C.byref(out.c), _ptr(steps_out), _stream(stream)))


def cosmica_batch_spectrum(batch: int, items, n_items: int, exit: ExitBuffers, bins: cosmica_bins, J, sigma, hist,
                           lis: Optional[cosmica_lis] = None, stream=None) -> None:
    lp = C.byref(lis) if lis is not None else None
    _check(lib().cosmica_batch_spectrum(batch, items, n_items, C.byref(exit.c), lp, C.byref(bins), _ptr(J),
                                        _ptr(sigma), _ptr(hist), _stream(stream)))


def cosmica_batch_spectrum_hist(batch: int, items, n_items: int, bins: cosmica_bins, hist, J, sigma,
                                lis: Optional[cosmica_lis] = None, stream=None) -> None:
    lp = C.byref(lis) if lis is not None else None
    _check(lib().cosmica_batch_spectrum_hist(batch, items, n_items, lp, C.byref(bins), _ptr(hist), _ptr(J),
                                             _ptr(sigma), _stream(stream)))


def cosmica_autotune(batch: int, items, n_items: int):
    t = cosmica_tuning()
    rate = C.c_double()
    _check(lib().cosmica_autotune(batch, items, n_items, C.byref(t), C.byref(rate)))
    return t, rate.value


def cosmica_last_error() -> str:
    return lib().cosmica_last_error().decode()


def cosmica_launch_count() -> int:
    return int(lib().cosmica_launch_count())


# -------------------------------------------------------------- server API --
def cosmica_server_create(mem_budget: int, precision: int = PREC_MIXED, budget_steps: int = 0) -> int:
    h = P()
    _check(lib().cosmica_server_create(int(mem_budget), int(precision), int(budget_steps), C.byref(h)))
    return h.value


def cosmica_server_destroy(h: int) -> None:
    lib().cosmica_server_destroy(h)


class Request:
    """A spectrum request with its host arrays kept alive."""

    def __init__(self, params: cosmica_params, species: cosmica_species, T_in, n_per_energy, seed: int,
                 bins: cosmica_bins):
        self.T = (C.c_double * len(T_in))(*[float(t) for t in T_in])
        self.N = (C.c_uint32 * len(T_in))(*[int(x) for x in n_per_energy])
        self.c = cosmica_request(params, species, C.cast(self.T, C.c_void_p), C.cast(self.N, C.c_void_p),
                                 len(T_in), int(seed), bins)
        self.n_energies = len(T_in)
        self.nbins = bins.nbins


def cosmica_server_submit(srv: int, req: Request) -> int:
    t = C.c_uint64()
    _check(lib().cosmica_server_submit(srv, C.byref(req.c), C.byref(t)))
    return t.value


class Result:
    def __init__(self, n_energies: int, nbins: int):
        import numpy as np
        self.J = np.zeros(n_energies)
        self.sigma = np.zeros(n_energies)
        self.hist = np.zeros((n_energies, nbins + 3), dtype=np.uint64)
        self.c = cosmica_result(self.J.ctypes.data, self.sigma.ctypes.data, self.hist.ctypes.data, 0, 0, 0, 0)

    @property
    def steps(self):
        return self.c.steps

    @property
    def latency(self):
        return self.c.t_done - self.c.t_submit


def cosmica_server_poll(srv: int, ticket: int, res: Result) -> bool:
    st = lib().cosmica_server_poll(srv, ticket, C.byref(res.c))
    if st == ERR_BUSY:
        return False
    _check(st)
    return True


def cosmica_server_wait(srv: int, ticket: int, res: Result, timeout_ms: int = 600_000) -> None:
    _check(lib().cosmica_server_wait(srv, ticket, int(timeout_ms), C.byref(res.c)))


def cosmica_server_stats_get(srv: int) -> dict:
    st = cosmica_server_stats()
    _check(lib().cosmica_server_stats_get(srv, C.byref(st)))
    return {f: getattr(st, f) for f, _ in cosmica_server_stats._fields_}


# --------------------------------------------------------------- debug API --
def cosmica_debug_philox(ctr, k0: int, k1: int, out, stream=None):
    _check(lib().cosmica_debug_philox(ctr.numel() // 4, _ptr(ctr), k0, k1, _ptr(out), _stream(stream)))


def cosmica_debug_curand_philox(seed: int, subseq, offset, out, stream=None):
    _check(lib().cosmica_debug_curand_philox(subseq.numel(), seed, _ptr(subseq), _ptr(offset), _ptr(out),
                                             _stream(stream)))


def cosmica_debug_normals64(seed: int, pid0: int, n: int, step: int, z, stream=None):
    _check(lib().cosmica_debug_normals64(seed, pid0, n, step, _ptr(z), _stream(stream)))


def cosmica_debug_normals32(seed: int, pid0: int, n: int, step: int, z, words=None, stream=None):
    _check(lib().cosmica_debug_normals32(seed, pid0, n, step, _ptr(z), _ptr(words), _stream(stream)))


FN_CODES = {"exp": 0, "log": 1, "sin": 2, "cos": 3, "tanh": 4, "atan": 5}


def cosmica_debug_fn64(name: str, x, y, stream=None):
    _check(lib().cosmica_debug_fn64(FN_CODES[name], x.numel(), _ptr(x), _ptr(y), _stream(stream)))


def cosmica_debug_eval(model: int, species: cosmica_species, precision: int, states, out, stream=None):
    _check(lib().cosmica_debug_eval(model, C.byref(species), precision, states.shape[0], _ptr(states), _ptr(out),
                                    _stream(stream)))


def exported_symbols():
    """Names declared in the public headers, for the symbol-export test."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = []
    for h in ("cosmica.h", "cosmica_debug.h"):
        txt = open(os.path.join(root, "include", h)).read()
        names += re.findall(r"^\s*(?:const\s+char|void|uint64_t|cosmica_status)\s*\**\s*(cosmica_\w+)\s*\(",
                            txt, flags=re.M)
    return sorted(set(names))
