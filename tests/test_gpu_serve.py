"""Continuous-batching server (cosmica_server_*): requests of different sizes
are admitted by device memory while others run, in-flight particles stay
resident (suspended exactly between quanta), and every result is the same
alone and in the mix -- bit for bit, since a path depends only on
(seed, pid, parameters) and the histogram is integer."""
import time

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import gpu_run, gpu_spectrum, torch

pytestmark = pytest.mark.gpu

BINS = cz.make_bins(0.1, 1000.0, 256)


def _req(p, sp, T, n, seed, prec=cz.PREC_MIXED):
    return cz.Request(cz.make_params(dict(p, max_steps=3_000_000), prec), cz.make_species(sp), T, n, seed, BINS)


def _mix(rng, k):
    sets = W.config3_param_sets()
    out = []
    for i in range(k):
        p = sets[int(rng.integers(0, 64))]
        sp = [W.PROTON, W.HELIUM4, W.ELECTRON][int(rng.integers(0, 3))]
        nE = int(rng.integers(2, 6))
        T = sorted(float(x) for x in np.exp(rng.uniform(np.log(0.2), np.log(50.0), nE)))
        n = [int(x) for x in rng.integers(1, 400, nE)]
        out.append((p, sp, T, n, 5000 + i))
    return out


def _run(srv, reqs, stagger_s=0.0):
    tickets = []
    for r in reqs:
        tickets.append(cz.cosmica_server_submit(srv, r))
        if stagger_s:
            time.sleep(stagger_s)
    res = []
    for r, t in zip(reqs, tickets):
        out = cz.Result(r.n_energies, r.nbins)
        cz.cosmica_server_wait(srv, t, out, timeout_ms=600_000)
        res.append(out)
    return res


def test_alone_equals_in_mix_bitwise():
    rng = np.random.default_rng(0)
    mix = _mix(rng, 8)
    target = mix[3]
    srv = cz.cosmica_server_create(2 << 30, cz.PREC_MIXED, budget_steps=512)
    alone = _run(srv, [_req(*target)])[0]
    many = _run(srv, [_req(*m) for m in mix], stagger_s=0.002)
    st = cz.cosmica_server_stats_get(srv)
    cz.cosmica_server_destroy(srv)
    inmix = many[3]
    assert np.array_equal(alone.hist, inmix.hist)
    assert np.array_equal(alone.J, inmix.J, equal_nan=True) and np.array_equal(alone.sigma, inmix.sigma, equal_nan=True)
    assert alone.steps == inmix.steps > 0
    assert st["quanta"] > 2 and st["completed"] == 9
    for r, m in zip(many, mix):
        assert r.hist.sum() == sum(m[3])


@pytest.mark.parametrize("prec", [cz.PREC_MIXED, cz.PREC_MIXED_F64ACC])
def test_server_equals_batched_path(prec):
    """The same request through cosmica_propagate (persistent batched kernel) and through
    the server (suspended and resumed every 256 steps) gives the same histogram."""
    p, sp, T, n, seed = W.config3_param_sets()[7], W.HELIUM4, [0.3, 2.0, 20.0], [150, 90, 61], 99
    srv = cz.cosmica_server_create(1 << 30, prec, budget_steps=256)
    r = _run(srv, [_req(p, sp, T, n, seed, prec)])[0]
    cz.cosmica_server_destroy(srv)
    job = W.Job(dict(p, max_steps=3_000_000), sp, T, n, seed, bins=W.Bins(0.1, 1000.0, 256))
    g, out, m = gpu_run(job, precision=prec)
    H, J, S = gpu_spectrum(job, out)
    m.close()
    assert np.array_equal(r.hist, H)
    assert np.allclose(r.J, J, rtol=1e-14, atol=0)


def test_admission_by_memory_and_overlap():
    srv_fixed = cz.cosmica_server_create(64 << 20, cz.PREC_MIXED, budget_steps=1024)
    cap = cz.cosmica_server_stats_get(srv_fixed)["arena_capacity"]
    cz.cosmica_server_destroy(srv_fixed)
    # a budget whose exit arena holds ~1.5 of these requests: they must queue
    per = 49
    sets = W.config3_param_sets()
    big = int(cap * 0.6)
    srv = cz.cosmica_server_create((64 << 20) - (cap - int(1.5 * big)) * per, cz.PREC_MIXED, budget_steps=1024)
    cap2 = cz.cosmica_server_stats_get(srv)["arena_capacity"]
    assert big <= cap2 < 2 * big
    reqs = [_req(sets[i], W.PROTON, [30.0, 60.0], [big // 2, big - big // 2], 700 + i) for i in range(3)]
    res = _run(srv, reqs)
    # a request that can never fit is rejected at submission
    with pytest.raises(cz.CosmicaError) as e:
        cz.cosmica_server_submit(srv, _req(sets[0], W.PROTON, [1.0], [cap2 + 1], 1))
    assert e.value.status == cz.ERR_INVALID
    st = cz.cosmica_server_stats_get(srv)
    cz.cosmica_server_destroy(srv)
    t = [(r.c.t_submit, r.c.t_admit, r.c.t_done) for r in res]
    # only one fits at a time: each is admitted no earlier than its predecessor finished
    assert t[1][1] >= t[0][2] - 1e-6 and t[2][1] >= t[1][2] - 1e-6
    assert st["rejected"] == 1 and st["completed"] == 3


def test_arrivals_overlap_running_work():
    """A request arriving while another runs is admitted before the first finishes."""
    sets = W.config3_param_sets()
    srv = cz.cosmica_server_create(2 << 30, cz.PREC_MIXED, budget_steps=512)
    a = _req(sets[1], W.ELECTRON, [0.15, 0.3], [3000, 3000], 11)   # long: low-energy electrons
    b = _req(sets[2], W.PROTON, [10.0], [500], 12)
    ta = cz.cosmica_server_submit(srv, a)
    time.sleep(0.05)
    tb = cz.cosmica_server_submit(srv, b)
    ra, rb = cz.Result(2, BINS.nbins), cz.Result(1, BINS.nbins)
    cz.cosmica_server_wait(srv, tb, rb)
    cz.cosmica_server_wait(srv, ta, ra)
    cz.cosmica_server_destroy(srv)
    assert rb.c.t_admit < ra.c.t_done
    assert rb.c.t_done < ra.c.t_done    # the short request does not wait for the long one


def test_wait_timeout_and_poll_busy():
    sets = W.config3_param_sets()
    srv = cz.cosmica_server_create(1 << 30, cz.PREC_MIXED, budget_steps=256)
    t = cz.cosmica_server_submit(srv, _req(sets[3], W.ELECTRON, [0.12], [4000], 3))
    res = cz.Result(1, BINS.nbins)
    assert cz.cosmica_server_poll(srv, t, res) is False
    with pytest.raises(cz.CosmicaError) as e:
        cz.cosmica_server_wait(srv, t, res, timeout_ms=1)
    assert e.value.status == cz.ERR_TIMEOUT
    cz.cosmica_server_wait(srv, t, res)
    assert res.hist.sum() == 4000
    with pytest.raises(cz.CosmicaError):
        cz.cosmica_server_poll(srv, t, res)    # the ticket was released
    cz.cosmica_server_destroy(srv)


def test_server_runs_extended_heliospheres_like_the_batched_path():
    """Requests with radial shells or a squashed heliosphere, served together with a basic
    one (the quantum then runs the extended kernel variant for all of them), give the
    histograms of the batched path."""
    shells = W.shell_params(W.solar_cycle_series(), rotation=60)
    squashed = W.params(R_ts=85.0, R_out=122.0, **W.SQUASHED)
    basic = W.config3_param_sets()[3]
    cases = [(shells, W.PROTON, [0.3, 3.0], [120, 80], 71), (squashed, W.HELIUM4, [0.5, 5.0], [90, 60], 72),
             (basic, W.ELECTRON, [1.0, 10.0], [70, 50], 73)]
    srv = cz.cosmica_server_create(1 << 30, cz.PREC_MIXED, budget_steps=512)
    res = _run(srv, [_req(p, sp, T, n, seed) for (p, sp, T, n, seed) in cases])
    cz.cosmica_server_destroy(srv)
    for (p, sp, T, n, seed), r in zip(cases, res):
        job = W.Job(dict(p, max_steps=3_000_000), sp, T, n, seed, bins=W.Bins(0.1, 1000.0, 256))
        g, out, m = gpu_run(job, precision=cz.PREC_MIXED)
        H, J, S = gpu_spectrum(job, out)
        m.close()
        assert np.array_equal(r.hist, H)
        assert np.allclose(r.J, J, rtol=1e-14, atol=0)


def test_server_rejects_the_energy_form():
    srv = cz.cosmica_server_create(1 << 28, cz.PREC_MIXED)
    with pytest.raises(cz.CosmicaError):
        cz.cosmica_server_submit(srv, _req(W.params(formulation=1.0), W.PROTON, [1.0], [10], 1))
    cz.cosmica_server_destroy(srv)
