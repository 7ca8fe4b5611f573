#!/usr/bin/env python3
"""Benchmark of the COSMICA hot path on GB300: SDE steps/s and spectra/s.

One bench "step" = one pass of the whole hot path over one batch of synthetic
input: work expansion into the device queue, the persistent propagation
launch (RNG, coefficients, Euler-Maruyama until every path exits), the
warp-aggregated histogram and the spectrum kernel.

Default workload (--workload c3, the largest single-GPU configuration): the
batched persistent launch over 64 heliospheres (K0, tilt, polarity and slow
wind drawn from their ranges, termination shock at 85 AU with x0.5 diffusion
beyond, boundary at 122 AU) x {proton, He-4, electron} x 30 energies with
uneven counts of 1e3-5e4 quasi-particles (7.4e7 in all, 192 spectra), mixed
precision (FP32 coefficients and normals, compensated FP32 accumulation,
exact boundary test), autotuned launch shape, CUDA-graph replay.  Beside the
throughput the line carries:
  * spectrum_error: the mixed spectra of twelve items of the workload against
    the FP64 CPU oracle's results for the same quasi-particles (stored by
    tests/golden/make_c3_golden.py), per item |dJ|/J and |dJ|/sigma;
  * fp64_plain: the plain FP64 GPU path (one thread per particle) and the
    mixed path timed on the same stratified sample of the workload;
  * serving: the continuous-batching server under Poisson request streams at
    0.5x and 0.8x of its measured capacity (p50/p99 latency, spectra/s);
  * cpu_baseline: the FP64 oracle on the host cores (all cores and one core)
    on stratified samples;
  * config2: config 2 (one heliosphere, 30 energies x 20 000 protons) timed
    beside it, a workload bound by its slowest paths rather than by issue.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run.  Default (--scaling strong): one
workload partitioned across the ranks by contiguous ranges of the global
particle index, histograms merged by one all-reduce per pass.  --scaling
weak: every rank propagates its own copy with disjoint particle identities.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_06319_gb300 import workloads as W  # noqa: E402
from paper_2502_06319_gb300.sharding import items_of, merge_histograms, partition, reduce_timing  # noqa: E402

METRIC = "SDE steps/s & spectra/s, FP32-batched vs plain FP64 GPU at <=0.5% spectrum error"
GOLDEN_C3 = os.path.join(ROOT, "tests", "golden", "oracle_c3_items.json")

# Algorithmic work of one mixed-precision step of the full model (drift and
# wavy sheet on), tallied from the source of the step (model32.cuh and the step
# of k_mixed.cu), each operation one issue slot: FP32 add/mul/fma (normals 15,
# coefficients 177, update 14, compensated accumulation 50, finiteness 4), SFU
# operations (normals 7, coefficients 23, sqrt(dt) 1), integer operations of
# the Philox block and the uniform mapping (66), and the comparisons of min/max,
# boundaries and exit tests (14).  A termination shock adds 9 FP32 + 2 SFU.
ALG_INST_PER_STEP = {"fp32": 260, "sfu": 31, "int_rng": 66, "compare": 14}
ALG_INST_TS = {"fp32": 9, "sfu": 2}
SM_LANES_PER_CLK = 128      # 4 SMSPs x 32 lanes: one warp instruction per SMSP per clock

# DRAM bytes (read + write) of the propagation launch per quasi-particle, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the batched workload at a
# reduced count; the bytes are the work-item reads and exit-record writes, so they scale
# with the particles of a launch (commands in profiles/).  They describe the kernel built
# from the sources whose SHA-256 is recorded; any other build reports traffic null.
TRAFFIC = {"c3": {"bytes_per_particle": 257347072 / 3715361,   # 57 048 064 read + 200 299 008 written, 5 % scale
                  "sources_sha256": "0d7d8d1018f6be1449eebf55aee1e53dcea69fce6e02098f038d1653968b5cda"}}
KERNEL_SOURCES = ("common.cuh", "philox.cuh", "model32.cuh", "mixed_state.cuh", "k_mixed.cu")


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2502_06319_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "shells", "squashed", "orbit"],
                    help="c3 (default): 64 heliospheres x 3 species x 30 energies, batched; shells: 13 "
                         "monthly observations of a 15-shell time-dependent heliosphere (Sec. II.B), proton + "
                         "He-4, batched like config 3; squashed: config 3 with the nose-squashed shock and outer "
                         "boundary (Sec. II.B); c4: the serving bench alone; orbit: config 2's heliosphere seen from a "
                         "detection point moving along a synthetic polar orbit (cosmica_propagate_orbit, Sec. IV.A)")
    ap.add_argument("--scaling", default="strong", choices=["strong", "weak"],
                    help="N > 1: partition one workload (strong) or give every rank a copy (weak)")
    ap.add_argument("--c4-requests", type=int, default=24, help="requests per serving run (--workload c4)")
    ap.add_argument("--serve-requests", type=int, default=60,
                    help="requests per load level of the serving key (0: no serving key)")
    ap.add_argument("--c3-scale", type=float, default=1.0, help="scale of config-3 particle counts")
    ap.add_argument("--scale", type=float, default=1.0, help="scale of config-1/2 particles per energy")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shape instead of the autotuner")
    ap.add_argument("--tuning", default="", help="fixed launch shape 'block,blocks_per_sm,compact_period' "
                                                  "instead of the autotuner")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_f64acc", "fp64"],
                    help="mixed: FP32 step with compensated FP32 (float-float) accumulation")
    ap.add_argument("--formulation", default="momentum", choices=["momentum", "energy"],
                    help="momentum form (Eq. 5-6, the method) or the energy form of Eq. 1 with loss weights "
                         "(configs 1-2 only)")
    ap.add_argument("--e2e-steps", type=int, default=2, help="passes timed end to end on the host")
    ap.add_argument("--fp64-sample", type=int, default=46080,
                    help="quasi-particles of the stratified sample the plain FP64 path is timed on (0: skip)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-c2", action="store_true",
                    help="skip the config-2 key of the default line (30 energies x 20 000 protons, tail-bound)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="quasi-particles of the oracle's stratified sample (all cores; reference arm: per step)")
    ap.add_argument("--probe-latency", action="store_true",
                    help="instead of the bench: the step latency of a lone path (one warp of config-1 "
                         "protons at 0.1 GeV, so the longest of 32 paths sets the time) and of few warps")
    return ap.parse_args()


def probe_latency(cz, torch):
    """Step latency when few warps are resident, the regime that ends every launch: time of a
    launch / steps of its longest path, for 32 (one warp) up to 152 x 32 x 16 particles."""
    p = W.params()
    b = cz.cosmica_batch_create([cz.make_params(p, cz.PREC_MIXED)], [cz.make_species(W.PROTON)])
    stream = torch.cuda.Stream()
    res = []
    for n in (32, 152 * 32, 152 * 32 * 16):
        items = cz.make_items([(0, 0, 0.1, n, 0, 11)])
        out = cz.ExitBuffers(n)
        steps = torch.zeros(1, dtype=torch.int64, device="cuda")
        tune = cz.cosmica_tuning(128, 0, 0, 0, 1)
        for _ in range(2):      # the second run is timed
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                cz.cosmica_batch_run(b, items, 1, out, tuning=tune, steps_out=steps, stream=stream)
                e1.record(stream)
            stream.synchronize()
        ms = e0.elapsed_time(e1)
        mx = int(out.numpy()["steps"].max())
        res.append({"particles": n, "ms": ms, "longest_path_steps": mx, "ns_per_step_of_longest": ms * 1e6 / mx,
                    "steps_per_s": int(steps.item()) / (ms * 1e-3)})
    cz.cosmica_batch_destroy(b)
    print(json.dumps({"probe": "lone-path step latency, config-1 protons at 0.1 GeV, mixed precision",
                      "runs": res}), flush=True)


def workload(args):
    """Jobs (one per spectrum) of the chosen configuration."""
    if args.workload == "orbit":
        raise SystemExit("--workload orbit is timed by our arm only (orbit_bench); the reference arm "
                         "times the batched workloads")
    if args.workload == "c4":
        return [r.job for r in W.config4(n_requests=args.c4_requests)], "config4 request sample"
    if args.workload == "c1":
        n = max(1, int(round(5000 * args.scale)))
        return [W.config1(n)], f"config1: full model, proton, 10 energies x {n}"
    if args.workload == "c2":
        n = max(1, int(round(20000 * args.scale)))
        return [W.config2(n)], f"config2: full model, proton, 30 energies x {n}"
    if args.workload == "squashed":
        jobs = W.config3(scale=args.c3_scale, geometry=W.SQUASHED)
        return jobs, (f"squashed: config3 (64 heliospheres x 3 species x 30 energies) with the nose-squashed "
                      f"shock (85 AU nose, x1.35 tail, x1.15 flank) and boundary (122 AU, x1.6, x1.25), "
                      f"scale {args.c3_scale}")
    if args.workload == "shells":
        jobs = W.config_shells(scale=args.c3_scale)
        return jobs, (f"shells: 13 Carrington rotations x 15 radial shells (synthetic solar cycle, seed 20250212) "
                      f"x {{proton, He-4}} x 30 energies, counts 1e3-5e4 (scale {args.c3_scale})")
    jobs = W.config3(scale=args.c3_scale)
    return jobs, (f"config3: 64 heliospheres (K0 5-30 AU^2/day, tilt 5-75 deg, A +-, slow wind 300-500 km/s; "
                  f"shock 85 AU, boundary 122 AU) x {{p, He-4, e-}} x 30 energies 0.1-100 GeV/n, counts "
                  f"1e3-5e4 log-uniform (scale {args.c3_scale})")


def stratified(items, n_target: int):
    """A sample of about n_target quasi-particles spread over the whole item list: the
    first m = n_target // n_items particles of every item when that is >= 1, else the
    first particle of every k-th item.  Returns (sample items, description)."""
    nI = len(items)
    if n_target >= nI:
        m = n_target // nI
        smp = [(pi, si, T, min(n, m), fp, sd) for (pi, si, T, n, fp, sd) in items[:] if n > 0]
        return smp, f"the first {m} quasi-particles of each of the {nI} items"
    k = max(1, nI // max(1, n_target))
    smp = [(pi, si, T, 1, fp, sd) for (pi, si, T, n, fp, sd) in items[::k] if n > 0]
    return smp, f"the first quasi-particle of every {k}-th of the {nI} items"


def cpu_baseline(params, species, items, n_target: int, threads: int = 0):
    """The FP64 oracle as it stands, on the host cores, on a stratified sample of the workload."""
    from oracle import oracle as O
    O.build()
    threads = threads or O.max_threads()
    smp, how = stratified(items, n_target)
    prm, spc, T, pid, seed = [], [], [], [], []
    for (pi, si, T_, n, fp, sd) in smp:
        prm += [pi] * n
        spc += [si] * n
        T += [T_] * n
        pid += range(fp, fp + n)
        seed += [sd] * n
    t0 = time.perf_counter()
    out = O.run_particles(params, species, np.array(prm, np.uint32), np.array(spc, np.uint32),
                          np.array(T, np.float64), np.array(pid, np.uint64), np.array(seed, np.uint64),
                          threads=threads)
    dt = time.perf_counter() - t0
    steps = int(out["steps"].astype(np.int64).sum())
    return {"value": steps / dt, "unit": "steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(T)} quasi-particles ({how}), {steps} steps in {dt:.1f} s", "seconds": dt,
            "steps": steps}


def default_cpu_sample(args, n_items: int, reference: bool) -> int:
    if args.cpu_sample:
        return args.cpu_sample
    if args.workload in ("c1", "c2"):
        return n_items * (600 if reference else 1500)
    return n_items * (1 if reference else 2)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on this machine's host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    jobs, desc = workload(args)
    params, species, items = items_of(jobs, 0)
    sample = default_cpu_sample(args, len(items), reference=True)
    for _ in range(max(0, args.warmup)):
        cpu_baseline(params, species, items, sample)
    secs, steps = 0.0, 0
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(params, species, items, sample)
        secs += cb["seconds"]; steps += cb["steps"]
    v = steps / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "sample_particles_per_step": sample},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_bench(cz, prec, n_cap: int, n_load: int, loads=(0.5, 0.8), offered=None):
    """The continuous-batching server (config 4 requests) under Poisson streams: capacity with
    n_cap requests queued at once, then n_load requests at each fraction of that capacity
    (and, if given, at the offered rate of config 4)."""
    reqs = W.config4(n_requests=n_cap + n_load * (len(loads) + (1 if offered else 0)) + 2)
    bins = cz.make_bins(0.1, 1000.0, 512)

    def make(r):
        j = r.job
        return cz.Request(cz.make_params(j.params, prec), cz.make_species(j.species), j.T_in, j.n_per_energy,
                          j.seed, bins)

    def run(batch, arrivals):
        srv = cz.cosmica_server_create(48 << 30, prec, budget_steps=4096)
        t0 = time.perf_counter()
        tickets = []
        for (r, ta) in zip(batch, arrivals):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append((cz.cosmica_server_submit(srv, make(r)), r))
        lat, steps = [], 0
        for t, r in tickets:
            res = cz.Result(len(r.job.T_in), 512)
            cz.cosmica_server_wait(srv, t, res, timeout_ms=3_600_000)
            lat.append(res.latency)
            steps += res.steps
        wall = time.perf_counter() - t0
        st = cz.cosmica_server_stats_get(srv)
        cz.cosmica_server_destroy(srv)
        return {"wall_s": wall, "steps": steps, "lat": lat, "quanta": st["quanta"]}

    nE = np.mean([len(r.job.T_in) for r in reqs[2:]])
    # per request: parameters + species + energies/counts + queue slices up; J, sigma, histogram down
    h2d = int(232 + 16 + nE * (8 + 4 + 48 + 8))
    d2h = int(nE * (16 + (512 + 3) * 8))
    run(reqs[:2], [0.0, 0.0])                          # warm-up (module load, first-launch costs)
    pos = 2
    cap = run(reqs[pos:pos + n_cap], [0.0] * n_cap)    # all queued at once: capacity
    pos += n_cap
    cap_rps = n_cap / cap["wall_s"]
    out = {"requests": "config4 stream (seed 20250211): 1 heliosphere x 1 species x 4-30 energies x 2e3-1e5 "
                       "quasi-particles per request", "server": "continuous batching, 4096 steps/lane/quantum",
           "h2d_bytes_per_request": h2d, "d2h_bytes_per_request": d2h,
           "capacity": {"requests": n_cap, "requests_per_s": cap_rps, "spectra_per_s": cap_rps,
                        "steps_per_s": cap["steps"] / cap["wall_s"], "quanta": cap["quanta"]}}
    rng = np.random.default_rng(20250211)
    levels = [(f"load_{f}", f * cap_rps) for f in loads] + ([("offered", offered)] if offered else [])
    for name, rate in levels:
        arr = np.cumsum(rng.exponential(1.0 / rate, n_load))
        rr = run(reqs[pos:pos + n_load], arr)
        pos += n_load
        lat = np.sort(rr["lat"])
        out[name] = {"rate_rps": rate, "requests": n_load, "p50_s": float(np.percentile(lat, 50)),
                     "p99_s": float(np.percentile(lat, 99)), "spectra_per_s": n_load / rr["wall_s"],
                     "steps_per_s": rr["steps"] / rr["wall_s"]}
    return out


def spectrum_error(items_spec, J, S):
    """Mixed spectra of the stored items against the FP64 oracle's (same quasi-particles)."""
    if not os.path.exists(GOLDEN_C3):
        return None
    g = json.load(open(GOLDEN_C3))
    key = {(it[4], it[3]): k for k, it in enumerate(items_spec)}     # (first_pid, n) -> row
    rows = []
    for rec in g["items"]:
        k = key.get((rec["first_pid"], rec["n"]))
        if k is None:
            return None
        d = J[k] - rec["J"]
        rows.append({"item": k, "species": rec["species"], "T": rec["T"], "n": rec["n"],
                     "tilt_deg": round(rec["tilt_deg"], 1), "polarity": int(rec["polarity"]),
                     "rel": d / rec["J"], "sigmas": abs(d) / math.hypot(S[k], rec["sigma"])})
    return {"vs": "FP64 CPU oracle, same quasi-particles (tests/golden/oracle_c3_items.json)",
            "items": len(rows), "max_abs_rel": max(abs(r["rel"]) for r in rows),
            "max_sigmas": max(r["sigmas"] for r in rows),
            "within_0.5pct_and_3sigma": all(abs(r["rel"]) <= 0.005 and r["sigmas"] <= 3.0 for r in rows),
            "per_item": rows}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def orbit_bench(args, cz, torch, prec, local):
    """The moving detection point (Sec. IV.A): config 2's heliosphere and energies, each energy's
    sample split among the positions of a synthetic polar orbit, through cosmica_propagate_orbit and
    cosmica_spectrum; W warm-up and K timed passes (CUDA events, L2 flushed before each), then passes
    timed end to end on the host."""
    n = max(1, int(round(20000 * args.scale)))
    job = W.config2(n)
    orbit = W.polar_orbit()
    model = cz.Model(cz.make_params(job.params, prec))
    sp = cz.make_species(job.species)
    bins = cz.make_bins(job.bins.P_min, job.bins.P_max, job.bins.n)
    nE, nb = len(job.T_in), job.bins.n
    out = cz.ExitBuffers(job.n_particles)
    J = torch.empty(nE, dtype=torch.float64, device="cuda")
    S = torch.empty_like(J)
    H = torch.empty(nE * (nb + 3), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()

    def one_pass(events=None):
        if events:
            events[0].record(stream)
        cz.cosmica_propagate_orbit(model.h, sp, job.T_in, job.n_per_energy, orbit, job.seed, out, stream=stream)
        if events:
            events[1].record(stream)
        cz.cosmica_spectrum(out, sp, job.T_in, bins, J, S, H, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_pass()
    stream.synchronize()
    steps_pass = int(out.steps.to(torch.int64).sum().item())      # the same every pass (fixed identities)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    launches0 = cz.cosmica_launch_count()
    ms, kern = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[2].record(stream)
            one_pass(ev[:2])
            ev[3].record(stream)
        ev[3].synchronize()
        ms.append(ev[2].elapsed_time(ev[3]))
        kern.append(ev[0].elapsed_time(ev[1]))
    launches = cz.cosmica_launch_count() - launches0
    torch.cuda.synchronize()
    clk = clocks.stop()
    J_h = torch.empty(nE, dtype=torch.float64, pin_memory=True)
    S_h = torch.empty(nE, dtype=torch.float64, pin_memory=True)
    H_h = torch.empty(nE * (nb + 3), dtype=torch.int64, pin_memory=True)
    e2e_s = 0.0
    n_e2e = max(1, args.e2e_steps)
    for _ in range(n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            one_pass()
            J_h.copy_(J, non_blocking=True)
            S_h.copy_(S, non_blocking=True)
            H_h.copy_(H, non_blocking=True)
        stream.synchronize()
        e2e_s += time.perf_counter() - t0
    model.close()
    nI = nE * len(orbit)                     # one work item per (position, energy)
    tot_ms, k_ms = sum(ms), sum(kern) / len(kern)
    steps_per_s = steps_pass * args.steps / (tot_ms * 1e-3)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    f_mhz = clk.get("sm_mhz") or 2070.0
    peak = SM_LANES_PER_CLK * sm_count * f_mhz * 1e6 / 1e12
    alg_total = sum(ALG_INST_PER_STEP.values())
    achieved = alg_total * steps_pass / (k_ms * 1e-3) / 1e12
    r_lo, r_hi = min(q[0] for q in orbit), max(q[0] for q in orbit)
    return {"metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64acc" if prec == cz.PREC_MIXED_F64ACC else ("f64" if prec == cz.PREC_FP64 else "f32+ff"),
            "data": "synthetic",
            "config": {"workload": f"orbit: config2's heliosphere (full model), proton, {nE} energies x {n} "
                                   f"quasi-particles, each energy's sample split over {len(orbit)} equal-time "
                                   f"positions of a synthetic polar orbit ({r_lo:.2f}-{r_hi:.2f} AU, inclination "
                                   f"80 deg)", "particles": job.n_particles, "precision": args.precision,
                       "l2": "flushed (256 MB write) before every timed step"},
            "spectra_per_s": args.steps / (tot_ms * 1e-3),
            "e2e": {"value": steps_pass * n_e2e / e2e_s, "unit": "steps/s",
                    "h2d_bytes_per_step": nI * 64 + 2 * (nI + 1) * 8 + nI * 4,
                    "d2h_bytes_per_step": 2 * nE * 8 + nE * (nb + 3) * 8, "passes": n_e2e},
            "gpu_launches": launches, "clocks": clk,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s",
                         "frac": achieved / peak, "traffic": None, "alg_inst_total": alg_total,
                         "kernel_ms_per_launch": k_ms, "algorithmic_bytes_per_step": 0.0}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2502_06319_gb300 import cosmica as cz

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU: the hot path has no CPU implementation")
    torch.cuda.set_device(local)
    if args.probe_latency:
        return probe_latency(cz, torch)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = {"mixed": cz.PREC_MIXED, "mixed_f64acc": cz.PREC_MIXED_F64ACC, "fp64": cz.PREC_FP64}[args.precision]

    if args.workload == "c4":
        launches0 = cz.cosmica_launch_count()
        clocks = Clocks(local)
        clocks.start()
        res = serve_bench(cz, prec if prec != cz.PREC_FP64 else cz.PREC_MIXED, args.c4_requests,
                          args.c4_requests, offered=200.0)
        clk = clocks.stop()
        v = res["capacity"]["steps_per_s"]
        line = {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world, "steps": args.c4_requests,
                "warmup": 2, "ms_per_step": 1e3 / res["capacity"]["requests_per_s"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64acc" if prec == cz.PREC_MIXED_F64ACC else "f32+ff",
                "data": "synthetic", "config": {"workload": "config4: Poisson request stream (seed 20250211), "
                                                "1 heliosphere x 1 species x 4-30 energies x 2e3-1e5 particles",
                                                "step": "one request (= one spectrum)"},
                "spectra_per_s": res["capacity"]["requests_per_s"], "serving": res,
                "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": res["h2d_bytes_per_request"],
                        "d2h_bytes_per_step": res["d2h_bytes_per_request"]},
                "gpu_launches": cz.cosmica_launch_count() - launches0, "clocks": clk}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    if args.workload == "orbit":
        if world > 1:
            raise SystemExit("--workload orbit runs on one GPU")
        line = orbit_bench(args, cz, torch, prec, local)
        print(json.dumps(line), flush=True)
        return

    jobs, desc = workload(args)
    energy = args.formulation == "energy"
    if energy:
        if args.workload not in ("c1", "c2"):
            raise SystemExit("--formulation energy applies to configs 1-2")
        for j in jobs:
            j.params = dict(j.params, formulation=1.0)
        desc += ", energy formulation (Eq. 1, loss-weighted Eq. 4)"
    strong = world > 1 and args.scaling == "strong"
    params, species, items_spec = items_of(jobs, 0 if strong else rank)
    if strong:
        share = partition(items_spec, world, rank)
        items_run = [piece for _, piece in share]
        exit_rows = [gi for gi, _ in share]
    else:
        items_run, exit_rows = items_spec, None
    n_total = sum(i[3] for i in items_run)
    n_spectra = len(jobs)
    nb = jobs[0].bins.n
    bins = cz.make_bins(jobs[0].bins.P_min, jobs[0].bins.P_max, nb)
    stream = torch.cuda.Stream()

    def make_batch(precision):
        return cz.cosmica_batch_create([cz.make_params(p, precision) for p in params],
                                       [cz.make_species(s) for s in species])

    arr = cz.make_items(items_run, exit_rows)
    nI = len(items_run)
    arr_spec = cz.make_items(items_spec)
    nS = len(items_spec)
    batch = make_batch(prec)
    if args.tuning:
        blk, bps, per = (int(x) for x in args.tuning.split(","))
        tune = cz.cosmica_tuning(blk, bps, per, 0, 1)
    elif args.no_autotune:
        tune = cz.cosmica_tuning(128, 0, 64, 0, 1)
    else:
        tune, _ = cz.cosmica_autotune(batch, arr, nI)
    tune.use_graph = 1
    out = cz.ExitBuffers(n_total, with_lw=energy)
    J = torch.empty(nS, dtype=torch.float64, device="cuda")
    S = torch.empty_like(J)
    H = torch.empty(nS * (nb + 3), dtype=torch.int64, device="cuda")
    steps_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2

    sp0 = cz.make_species(jobs[0].species)
    kernel_ms = []      # propagation launches alone, CUDA events on the launching stream

    def one_pass(b, t, time_kernel=False):
        if time_kernel:
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            k0.record(stream)
        cz.cosmica_batch_run(b, arr, nI, out, tuning=t, steps_out=steps_dev, stream=stream)
        if time_kernel:
            k1.record(stream)
            kernel_ms.append((k0, k1))
        if energy:   # loss-weighted Eq. 4 (items are the energies of one job, in exit order)
            cz.cosmica_spectrum_unbinned(out, sp0, jobs[0].T_in, jobs[0].n_per_energy, 1, J, S, stream=stream)
        else:
            # bin this rank's exit records into the rows of the whole item list
            cz.cosmica_batch_spectrum(b, arr_spec, nS, out, bins, J, S, H, stream=stream)
            if strong:
                merge_histograms(dist, H)       # NCCL all-reduce on the current (= launching) stream
                cz.cosmica_batch_spectrum_hist(b, arr_spec, nS, bins, H, J, S, stream=stream)

    def timed(b, t, warm, k):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                one_pass(b, t)
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ms, steps, launches = [], 0, cz.cosmica_launch_count()
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one_pass(b, t, time_kernel=True)
                e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            steps += int(steps_dev.item())
        launches = cz.cosmica_launch_count() - launches
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return ms, steps, launches

    clocks = Clocks(local)
    clocks.start()
    ms, steps_done, launches = timed(batch, tune, args.warmup, args.steps)
    clk = clocks.stop()
    kern_ms = sum(k0.elapsed_time(k1) for k0, k1 in kernel_ms)
    kern_launches = len(kernel_ms)
    tot_ms = sum(ms)
    tot_ms, steps_all = reduce_timing(dist, tot_ms, float(steps_done), device="cuda")
    steps_per_s = steps_all / (tot_ms * 1e-3)
    n_spec_all = n_spectra * (1 if strong else world)
    spectra_per_s = n_spec_all * args.steps / (tot_ms * 1e-3)
    Jm, Sm = J.cpu().numpy().copy(), S.cpu().numpy().copy()

    # end to end through the public API, timed on the host: each step the library copies the
    # step's inputs (work items, prefix sums) host -> device inside cosmica_batch_run, and the
    # spectrum and histogram are read back into pinned host memory
    J_h = torch.empty(nS, dtype=torch.float64, pin_memory=True)
    S_h = torch.empty(nS, dtype=torch.float64, pin_memory=True)
    H_h = torch.empty(nS * (nb + 3), dtype=torch.int64, pin_memory=True)
    e2e_steps, e2e_s = 0, 0.0
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            one_pass(batch, tune)
            J_h.copy_(J, non_blocking=True)
            S_h.copy_(S, non_blocking=True)
            H_h.copy_(H, non_blocking=True)
        stream.synchronize()
        e2e_s += time.perf_counter() - t0
        e2e_steps += int(steps_dev.item())
    e2e_s, e2e_steps = reduce_timing(dist, e2e_s, float(e2e_steps), device="cuda")
    h2d = nI * 64 + 2 * (nI + 1) * 8 + nI * 4 + nS * 40   # work items, prefix sums, queue order, spectrum items
    d2h = 2 * nS * 8 + nS * (nb + 3) * 8

    # accuracy: the mixed spectra of the stored items against the FP64 oracle
    err = spectrum_error(items_spec, Jm, Sm) if (args.workload == "c3" and args.c3_scale == 1.0
                                                 and not energy and rank == 0) else None

    # plain FP64 GPU path and the mixed path on the same stratified sample of the workload
    fp64 = None
    if not args.no_fp64 and args.fp64_sample > 0 and prec != cz.PREC_FP64 and world == 1:
        smp, how = stratified(items_spec, args.fp64_sample)
        arr_s = cz.make_items(smp)
        n_s = sum(i[3] for i in smp)
        out_s = cz.ExitBuffers(n_s, with_lw=energy)
        rates = {}
        for name, pr in (("fp64", cz.PREC_FP64), ("mixed", prec)):
            bb = make_batch(pr) if pr != prec else batch
            tt = None if pr == cz.PREC_FP64 else cz.cosmica_tuning(128, 0, 64, 0, 0)
            with torch.cuda.stream(stream):
                cz.cosmica_batch_run(bb, arr_s, len(smp), out_s, tuning=tt, steps_out=steps_dev, stream=stream)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cz.cosmica_batch_run(bb, arr_s, len(smp), out_s, tuning=tt, steps_out=steps_dev, stream=stream)
                e1.record(stream)
            e1.synchronize()
            rates[name] = (int(steps_dev.item()) / (e0.elapsed_time(e1) * 1e-3), e0.elapsed_time(e1))
            if bb is not batch:
                cz.cosmica_batch_destroy(bb)
        fp64 = {"sample": f"{n_s} quasi-particles ({how})", "steps_per_s": rates["fp64"][0],
                "ms": rates["fp64"][1], "mixed_steps_per_s_same_sample": rates["mixed"][0],
                "mixed_ms_same_sample": rates["mixed"][1],
                "mixed_over_fp64": rates["mixed"][0] / rates["fp64"][0],
                "accuracy": "FP64 GPU paths are bit-identical to the FP64 oracle (tests); the mixed spectra's error "
                            "against the oracle is spectrum_error"}

    # config 2 beside the headline: one heliosphere, 6e5 paths, bound by its slowest paths
    config2 = None
    if args.workload == "c3" and not args.no_c2 and world == 1 and prec == cz.PREC_MIXED:
        j2 = W.config2()
        p2, s2, it2 = items_of([j2], 0)
        b2 = cz.cosmica_batch_create([cz.make_params(p, prec) for p in p2], [cz.make_species(x) for x in s2])
        a2 = cz.make_items(it2)
        t2, _ = cz.cosmica_autotune(b2, a2, len(it2))
        t2.use_graph = 1
        o2 = cz.ExitBuffers(sum(i[3] for i in it2))
        J2 = torch.empty(len(it2), dtype=torch.float64, device="cuda")
        S2 = torch.empty_like(J2)
        H2 = torch.empty(len(it2) * (j2.bins.n + 3), dtype=torch.int64, device="cuda")
        bins2 = cz.make_bins(j2.bins.P_min, j2.bins.P_max, j2.bins.n)
        ms2, st2 = 0.0, 0
        for rep in range(5):          # 2 warm-up + 3 timed passes
            with torch.cuda.stream(stream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                cz.cosmica_batch_run(b2, a2, len(it2), o2, tuning=t2, steps_out=steps_dev, stream=stream)
                cz.cosmica_batch_spectrum(b2, a2, len(it2), o2, bins2, J2, S2, H2, stream=stream)
                e1.record(stream)
            e1.synchronize()
            if rep >= 2:
                ms2 += e0.elapsed_time(e1)
                st2 += int(steps_dev.item())
        cz.cosmica_batch_destroy(b2)
        rate2 = st2 / (ms2 * 1e-3)
        config2 = {"workload": "config2: full model, proton, 30 energies x 20000 (one heliosphere, 6e5 paths)",
                   "steps_per_s": rate2, "ms_per_pass": ms2 / 3, "spectra_per_s": 3 / (ms2 * 1e-3),
                   "issue_roofline_frac": sum(ALG_INST_PER_STEP.values()) * rate2 / 1e12 / (
                       SM_LANES_PER_CLK * torch.cuda.get_device_properties(local).multi_processor_count
                       * (clk.get("sm_mhz") or 2070.0) * 1e6 / 1e12),
                   "tuning": {"block": t2.block, "blocks_per_sm": t2.blocks_per_sm,
                              "compact_period": t2.compact_period},
                   "note": "bound by its slowest paths (a lone path's step), not by issue"}

    serving = None
    if args.serve_requests > 0 and world == 1 and prec != cz.PREC_FP64:
        serving = serve_bench(cz, prec, n_cap=max(8, args.serve_requests // 4), n_load=args.serve_requests)

    # roofline: algorithmic issue slots per step x steps/s against the SM issue rate
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    f_mhz = clk.get("sm_mhz") or 2070.0
    peak = SM_LANES_PER_CLK * sm_count * f_mhz * 1e6 / 1e12          # T inst/s
    alg = dict(ALG_INST_PER_STEP)
    if any(p.get("R_ts", 0.0) > 0.0 for p in params):
        for k, v in ALG_INST_TS.items():
            alg[k] += v
    alg_total = sum(alg.values())
    # achieved: algorithmic issue slots of one launch (tally x the launch's steps) / the launch's
    # average duration (CUDA events around the propagation call alone, this rank)
    achieved = alg_total * (steps_done / max(1, kern_launches)) / (kern_ms / max(1, kern_launches) * 1e-3) / 1e12
    traffic = None
    tr = TRAFFIC.get(args.workload)
    if (tr and tr["bytes_per_particle"] is not None and not energy and prec == cz.PREC_MIXED and not strong
            and tr["sources_sha256"] == kernel_sources_sha256()):
        traffic = tr["bytes_per_particle"] * n_total
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
            "traffic": traffic, "peak_basis": f"{SM_LANES_PER_CLK} lanes/clk/SM x {sm_count} SMs x "
                                              f"{f_mhz:.0f} MHz (median SM clock sampled under load)",
            "alg_inst_per_step": alg, "alg_inst_total": alg_total,
            "kernel_ms_per_launch": kern_ms / max(1, kern_launches),
            "algorithmic_bytes_per_step": 0.0}

    line = {"metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if strong else "weak", "vs_baseline": None,
            "dtype": "f32+ff" if prec == cz.PREC_MIXED else ("f32+f64acc" if prec == cz.PREC_MIXED_F64ACC else "f64"),
            "data": "synthetic",
            "config": {"workload": desc,
                       "particles": sum(i[3] for i in items_spec) if strong else n_total * world,
                       "particles_per_gpu": n_total, "spectra_per_step": n_spec_all,
                       "precision": args.precision, "formulation": args.formulation,
                       "tuning": {"block": tune.block, "blocks_per_sm": tune.blocks_per_sm,
                                  "compact_period": tune.compact_period, "queue_order": tune.queue_order,
                                  "graph": bool(tune.use_graph)},
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": (f"partition x{world} (pid ranges, histogram all-reduce)" if strong
                                       else f"replicas x{world}")},
            "spectra_per_s": spectra_per_s,
            "e2e": {"value": e2e_steps / e2e_s if e2e_s else None, "unit": "steps/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "passes": max(1, args.e2e_steps)},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "spectrum_error": err,
            "fp64_plain": fp64, "serving": serving, "config2": config2}
    if rank == 0 and not args.no_cpu and world == 1:
        n_all = default_cpu_sample(args, len(items_spec), reference=False)
        cb = cpu_baseline(params, species, items_spec, n_all)
        c1 = cpu_baseline(params, species, items_spec, max(1, n_all // 16), threads=1)
        line["cpu_baseline"] = {k: v for k, v in cb.items() if k in ("value", "unit", "cores", "kind", "sample")}
        line["cpu_baseline"]["single_thread"] = {k: v for k, v in c1.items()
                                                 if k in ("value", "unit", "cores", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    cz.cosmica_batch_destroy(batch)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
