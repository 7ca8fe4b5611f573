#!/usr/bin/env python3
"""Benchmark of the COSMICA hot path on GB300: SDE steps/s and spectra/s.

One bench "step" = one pass of the whole hot path over one batch of synthetic
input: work expansion into the device queue, the persistent propagation
launch (RNG, coefficients, Euler-Maruyama until every path exits), the
warp-aggregated histogram and the spectrum kernel.

Default workload (--workload c2): the full heliospheric model (Parker field,
two-speed wind, drifts, wavy current sheet, tilt 20 deg, qA > 0) for protons
at 30 log-spaced energies in 0.1-100 GeV with 20 000 quasi-particles each,
mixed precision (FP32 coefficients and normals, compensated FP32
accumulation, exact boundary test), batched persistent launch.  The plain
FP64 GPU path is timed on the same workload and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; each rank propagates its own
copy of the workload with disjoint particle identities (weak scaling, no
collective on the data path).
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
from paper_2502_06319_gb300.sharding import items_of, reduce_timing  # noqa: E402

METRIC = "SDE steps/s & spectra/s, FP32-batched vs plain FP64 GPU at <=0.5% spectrum error"

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

# DRAM bytes (read + write) of one propagation launch of the default workload (config 2),
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum; the command is in
# profiles/launches_bench_c2.md).  They describe the kernel built from the sources whose
# SHA-256 is recorded; any other build reports traffic null.
TRAFFIC_C2 = {"bytes_per_launch": 9298176,   # 4 887 552 read + 4 410 624 written
              "sources_sha256": "a6c707982578db0c9c3b43f0ef653237e84263566c8d3d549781281d557f7566"}
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
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "shells", "squashed"],
                    help="shells: 13 monthly observations of a 15-shell time-dependent heliosphere "
                         "(Sec. II.B), proton + He-4, batched like config 3; squashed: config 3 with "
                         "the nose-squashed shock and outer boundary (Sec. II.B)")
    ap.add_argument("--c4-requests", type=int, default=24, help="requests per serving run")
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
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--cpu-sample", type=int, default=0, help="particles per energy in the oracle sample")
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
    return jobs, f"config3: 64 heliospheres x 3 species x 30 energies, counts 1e3-5e4 (scale {args.c3_scale})"


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


def cpu_baseline(jobs, sample_per_energy: int):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload."""
    from oracle import oracle as O
    O.build()
    threads = O.max_threads()
    job = jobs[0]
    sel = []
    off = 0
    for n in job.n_per_energy:
        sel.extend(range(off, off + min(n, sample_per_energy)))
        off += n
    t0 = time.perf_counter()
    out = O.job_run(job, select=np.asarray(sel), threads=threads)
    dt = time.perf_counter() - t0
    steps = int(out["steps"].astype(np.int64).sum())
    return {"value": steps / dt, "unit": "steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(sel)} quasi-particles ({sample_per_energy} per energy of {job.name}), "
                      f"{steps} steps in {dt:.1f} s", "seconds": dt, "steps": steps}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on this machine's host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    jobs, desc = workload(args)
    sample = args.cpu_sample or (600 if args.workload != "c1" else 1500)
    if args.warmup > 0:
        cpu_baseline(jobs, max(2, sample // 10))
    vals, secs, steps = [], 0.0, 0
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(jobs, sample)
        vals.append(cb["value"]); secs += cb["seconds"]; steps += cb["steps"]
    v = steps / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "sample_per_energy": sample},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_bench(args, cz, torch):
    """Config 4: the continuous-batching server under a Poisson request stream."""
    import math as _m
    reqs = W.config4(n_requests=4 * args.c4_requests)
    prec = cz.PREC_MIXED if args.precision == "mixed" else cz.PREC_MIXED_F64ACC
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
        return {"wall_s": wall, "steps": steps, "lat": lat, "quanta": st["quanta"], "busy_s": st["busy_seconds"]}

    M = args.c4_requests
    nE = np.mean([len(r.job.T_in) for r in reqs[:M]])
    # per request: parameters + species + energies/counts + queue slices up; J, sigma, histogram down
    h2d = int(232 + 16 + nE * (8 + 4 + 48 + 8))
    d2h = int(nE * (16 + (512 + 3) * 8))
    # warm-up (module load, first-launch costs)
    run(reqs[:2], [0.0, 0.0])
    cap = run(reqs[:M], [0.0] * M)                     # all queued at once: capacity
    cap_rps = M / cap["wall_s"]
    out = {"h2d_bytes_per_request": h2d, "d2h_bytes_per_request": d2h,
           "capacity": {"requests_per_s": cap_rps, "steps_per_s": cap["steps"] / cap["wall_s"],
                        "quanta": cap["quanta"]}}
    rng = np.random.default_rng(20250211)
    for name, rate in (("load_0.5", 0.5 * cap_rps), ("load_0.8", 0.8 * cap_rps), ("offered_200", 200.0)):
        arr = np.cumsum(rng.exponential(1.0 / rate, M))
        rr = run(reqs[M:2 * M] if name != "offered_200" else reqs[2 * M:3 * M], arr)
        lat = np.sort(rr["lat"])
        out[name] = {"rate_rps": rate, "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                     "spectra_per_s": M / rr["wall_s"], "steps_per_s": rr["steps"] / rr["wall_s"]}
    return out, cap


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

    if args.workload == "c4":
        launches0 = cz.cosmica_launch_count()
        clocks = Clocks(local)
        clocks.start()
        res, cap = serve_bench(args, cz, torch)
        clk = clocks.stop()
        v = res["capacity"]["steps_per_s"]
        line = {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world, "steps": args.c4_requests,
                "warmup": 2, "ms_per_step": 1e3 / res["capacity"]["requests_per_s"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc" if args.precision != "mixed" else "f32+ff",
                "data": "synthetic", "config": {"workload": "config4: Poisson request stream (seed 20250211), "
                                                "1 heliosphere x 1 species x 4-30 energies x 2e3-1e5 particles",
                                                "server": "continuous batching, 4096 steps/lane/quantum, 48 GB budget",
                                                "step": "one request (= one spectrum)"},
                "spectra_per_s": res["capacity"]["requests_per_s"], "serving": res,
                "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": res["h2d_bytes_per_request"],
                        "d2h_bytes_per_step": res["d2h_bytes_per_request"]},
                "gpu_launches": cz.cosmica_launch_count() - launches0, "clocks": clk}
        if rank == 0:
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
    prec = {"mixed": cz.PREC_MIXED, "mixed_f64acc": cz.PREC_MIXED_F64ACC, "fp64": cz.PREC_FP64}[args.precision]
    params, species, items = items_of(jobs, rank)
    n_total = sum(i[3] for i in items)
    n_spectra = len(jobs)
    nb = jobs[0].bins.n
    bins = cz.make_bins(jobs[0].bins.P_min, jobs[0].bins.P_max, nb)
    stream = torch.cuda.Stream()

    def make_batch(precision):
        return cz.cosmica_batch_create([cz.make_params(p, precision) for p in params],
                                       [cz.make_species(s) for s in species])

    arr = cz.make_items(items)
    nI = len(items)
    batch = make_batch(prec)
    if args.tuning:
        blk, bps, per = (int(x) for x in args.tuning.split(","))
        tune = cz.cosmica_tuning(blk, bps, per, 0, 1)
    elif args.no_autotune:
        tune = cz.cosmica_tuning(128, 0, 64, 0, 1)
    else:
        tune, tune_rate = cz.cosmica_autotune(batch, arr, nI)
    tune.use_graph = 1
    out = cz.ExitBuffers(n_total, with_lw=energy)
    J = torch.empty(nI, dtype=torch.float64, device="cuda")
    S = torch.empty_like(J)
    H = torch.empty(nI * (nb + 3), dtype=torch.int64, device="cuda")
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
            cz.cosmica_batch_spectrum(b, arr, nI, out, bins, J, S, H, stream=stream)

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
    spectra_per_s = n_spectra * world * args.steps / (tot_ms * 1e-3)
    Jm = J.cpu().numpy().copy()

    # end to end through the public API, timed on the host: each step the library copies the
    # step's inputs (work items, prefix sums) host -> device inside cosmica_batch_run, and the
    # spectrum and histogram are read back into pinned host memory
    J_h = torch.empty(nI, dtype=torch.float64, pin_memory=True)
    S_h = torch.empty(nI, dtype=torch.float64, pin_memory=True)
    H_h = torch.empty(nI * (nb + 3), dtype=torch.int64, pin_memory=True)
    e2e_steps, e2e_s = 0, 0.0
    for it in range(1 + max(1, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            one_pass(batch, tune)
            J_h.copy_(J, non_blocking=True)
            S_h.copy_(S, non_blocking=True)
            H_h.copy_(H, non_blocking=True)
        stream.synchronize()
        dt = time.perf_counter() - t0
        if it > 0:
            e2e_s += dt
            e2e_steps += int(steps_dev.item())
    h2d = nI * 64 + 2 * (nI + 1) * 8 + nI * 4     # work items, two prefix-sum tables, queue order
    d2h = 2 * nI * 8 + nI * (nb + 3) * 8

    # plain FP64 GPU path on the same workload (one-thread-per-particle launch)
    fp64 = None
    if not args.no_fp64 and prec != cz.PREC_FP64:
        b64 = make_batch(cz.PREC_FP64)
        ms64, st64, _ = timed(b64, None, 1, 1)
        J64 = J.cpu().numpy().copy()
        fp64 = {"steps_per_s": st64 / (sum(ms64) * 1e-3), "ms_per_step": sum(ms64),
                "max_spectrum_rel_diff_mixed_vs_fp64": float(np.nanmax(np.abs(Jm / J64 - 1)))}
        cz.cosmica_batch_destroy(b64)

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
    if (args.workload == "c2" and args.scale == 1.0 and not energy and prec == cz.PREC_MIXED
            and TRAFFIC_C2["bytes_per_launch"] is not None
            and TRAFFIC_C2["sources_sha256"] == kernel_sources_sha256()):
        traffic = TRAFFIC_C2["bytes_per_launch"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
            "traffic": traffic, "peak_basis": f"{SM_LANES_PER_CLK} lanes/clk/SM x {sm_count} SMs x "
                                              f"{f_mhz:.0f} MHz (median SM clock sampled under load)",
            "alg_inst_per_step": alg, "alg_inst_total": alg_total,
            "kernel_ms_per_launch": kern_ms / max(1, kern_launches),
            "algorithmic_bytes_per_step": 0.0}

    line = {"metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff" if prec == cz.PREC_MIXED else
            ("f32+f64acc" if prec == cz.PREC_MIXED_F64ACC else "f64"), "data": "synthetic",
            "config": {"workload": desc, "particles_per_gpu": n_total, "spectra_per_step": n_spectra,
                       "precision": args.precision, "formulation": args.formulation, "tuning": {"block": tune.block,
                                                               "blocks_per_sm": tune.blocks_per_sm,
                                                               "compact_period": tune.compact_period,
                                                               "queue_order": tune.queue_order,
                                                               "graph": bool(tune.use_graph)},
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": f"weak x{world}"},
            "spectra_per_s": spectra_per_s,
            "e2e": {"value": e2e_steps / e2e_s if e2e_s else None, "unit": "steps/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "fp64_plain": fp64}
    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(jobs, args.cpu_sample or 1500).items()
                                if k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    cz.cosmica_batch_destroy(batch)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
