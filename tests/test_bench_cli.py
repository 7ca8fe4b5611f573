"""bench.py's command-line contract on the CPU: the reference arm (the FP64
oracle on the host cores) prints one JSON line with the keys the contract
names, only rank 0 prints, our arm refuses to run without a CUDA GPU instead
of falling back to the CPU, and the clock record of the timed region reports
the median SM clock and every throttle reason that was active."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*argv, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *argv], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _bench("--impl", "reference", "--steps", "2", "--warmup", "1", "--cpu-sample", "10")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["ms_per_step"] > 0 and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["scaling"] == "weak" and d["dtype"] == "f64" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_stay_silent():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-sample", "5", env={"RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_our_arm_fails_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _bench("--steps", "1", "--warmup", "0")
    assert r.returncode != 0
    assert "CUDA GPU" in (r.stdout + r.stderr)


def test_clock_record_from_a_fake_nvidia_smi():
    # the clock and throttle record of the timed region, parsed from nvidia-smi's CSV rows
    # (index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap);
    # no GPU and no nvidia-smi: the sampler's process is a stand-in that has already ended
    sys.path.insert(0, ROOT)
    import bench

    class Ended:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.Clocks(0)
    c.f.write("0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "0, 2055, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active\n"
              "0, 2070, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active\n"
              "garbage line\n")
    c.proc = Ended()
    rec = c.stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c = bench.Clocks(0)
    c.f.write("0, 1200, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active\n")
    c.proc = Ended()
    assert c.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_stratified_samples_span_the_whole_item_list():
    # the samples the plain FP64 path and the oracle baseline are timed on: the first m particles
    # of every non-empty item (capped at its count), or the first particle of every k-th item
    sys.path.insert(0, ROOT)
    import bench
    items = [(0, 0, 0.1 * (i + 1), n, 1000 * i, 7) for i, n in enumerate([5, 0, 1, 9, 3, 2, 8, 4])]
    smp, how = bench.stratified(items, 24)            # 24 // 8 = 3 per item
    assert [s[3] for s in smp] == [3, 1, 3, 3, 2, 3, 3] and "first 3" in how
    assert [s[4] for s in smp] == [0, 2000, 3000, 4000, 5000, 6000, 7000]   # identities kept
    smp, how = bench.stratified(items, 3)             # every 2nd item, one particle each
    assert [(s[4], s[3]) for s in smp] == [(0, 1), (2000, 1), (4000, 1), (6000, 1)] and "every 2-th" in how


def test_spectrum_error_maps_the_stored_items_onto_the_full_workload():
    # the twelve stored oracle items of config 3 must be found in today's config-3 item list by
    # (first particle identity, count) -- the input generator and the stored values agree -- and
    # the error record flags a deviation beyond 0.5 %
    sys.path.insert(0, ROOT)
    import bench
    from paper_2502_06319_gb300 import workloads as W
    _, _, items = W.items_of(W.config3(), 0)
    g = json.load(open(bench.GOLDEN_C3))
    J = [float("nan")] * len(items)
    S = [0.0] * len(items)
    key = {(it[4], it[3]): k for k, it in enumerate(items)}
    for rec in g["items"]:
        k = key[(rec["first_pid"], rec["n"])]
        assert abs(items[k][2] - rec["T"]) < 1e-12
        J[k], S[k] = rec["J"], rec["sigma"]
    e = bench.spectrum_error(items, J, S)
    assert e["items"] == 12 and e["max_abs_rel"] == 0.0 and e["within_0.5pct_and_3sigma"]
    k = key[(g["items"][0]["first_pid"], g["items"][0]["n"])]
    J[k] *= 1.006
    assert not bench.spectrum_error(items, J, S)["within_0.5pct_and_3sigma"]
