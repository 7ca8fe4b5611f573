"""Batched persistent launch: many (parameter set, species, energy) work items
with uneven counts in one launch fed by the device work queue.  A particle's
result depends only on (seed, pid, parameters, species, energy), so every item
of a batch must equal the same item propagated alone, bit for bit."""
import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import torch

pytestmark = pytest.mark.gpu


def _setup(precision, counts_seed=0):
    sets = W.config3_param_sets()[:3]
    species = [W.PROTON, W.HELIUM4, W.ELECTRON]
    T = [0.15, 1.5, 15.0, 80.0]
    rng = np.random.default_rng(counts_seed)
    items = []
    pid = 0
    for pi in range(3):
        for si in range(3):
            for T_ in T:
                n = int(rng.choice([0, 1, 17, 64, 150]))
                items.append((pi, si, T_, n, 1000 + pid, 777 + pi))
                pid += n
    params = [cz.make_params(dict(p, max_steps=2_000_000), precision) for p in sets]
    b = cz.cosmica_batch_create(params, [cz.make_species(s) for s in species])
    return sets, species, items, b


@pytest.mark.parametrize("precision", [cz.PREC_FP64, cz.PREC_MIXED])
def test_batch_items_equal_single_runs(precision):
    t = torch()
    sets, species, items, b = _setup(precision)
    arr = cz.make_items(items)
    total = sum(i[3] for i in items)
    out = cz.ExitBuffers(total)
    steps = t.zeros(1, dtype=t.int64, device="cuda")
    cz.cosmica_batch_run(b, arr, len(items), out, steps_out=steps)
    t.cuda.synchronize()
    g = out.numpy()
    assert int(steps.item()) == int(g["steps"].astype(np.int64).sum())
    off = 0
    for k, (pi, si, T_, n, fp, sd) in enumerate(items):
        if n == 0:
            continue
        single = cz.cosmica_batch_create([cz.make_params(dict(sets[pi], max_steps=2_000_000), precision)],
                                         [cz.make_species(species[si])])
        o1 = cz.ExitBuffers(n)
        cz.cosmica_batch_run(single, cz.make_items([(0, 0, T_, n, fp, sd)]), 1, o1)
        t.cuda.synchronize()
        s = o1.numpy()
        for key in ("r", "th", "ph", "lnP", "s", "steps", "status"):
            assert np.array_equal(g[key][off:off + n], s[key]), (k, key)
        assert np.all(g["item"][off:off + n] == k)
        cz.cosmica_batch_destroy(single)
        off += n
    cz.cosmica_batch_destroy(b)


def test_graph_replay_and_batch_spectrum():
    t = torch()
    sets, species, items, b = _setup(cz.PREC_MIXED, counts_seed=1)
    arr = cz.make_items(items)
    total = sum(i[3] for i in items)
    s = t.cuda.Stream()
    res, outs = [], []
    for rep in range(3):
        # all three buffers stay alive, so every replay writes to new addresses
        out = cz.ExitBuffers(total)
        outs.append(out)
        steps = t.zeros(1, dtype=t.int64, device="cuda")
        tune = cz.cosmica_tuning(128, 0, 64, 1, 1)
        with t.cuda.stream(s):
            cz.cosmica_batch_run(b, arr, len(items), out, tuning=tune, steps_out=steps, stream=s)
        s.synchronize()
        res.append((out.numpy(), int(steps.item())))
    for k in res[0][0]:
        assert np.array_equal(res[0][0][k], res[1][0][k]) and np.array_equal(res[0][0][k], res[2][0][k])
    assert res[0][1] == res[2][1] > 0
    nb = 512
    J = t.empty(len(items), dtype=t.float64, device="cuda")
    S = t.empty_like(J)
    H = t.empty(len(items) * (nb + 3), dtype=t.int64, device="cuda")
    cz.cosmica_batch_spectrum(b, arr, len(items), out, cz.make_bins(0.1, 1000.0, nb), J, S, H)
    t.cuda.synchronize()
    Hn = H.cpu().numpy().reshape(len(items), nb + 3)
    counts = np.array([i[3] for i in items])
    assert np.array_equal(Hn.sum(axis=1), counts)
    Jn = J.cpu().numpy()
    assert np.all(np.isnan(Jn[counts == 0])) and np.all(np.isfinite(Jn[counts > 0]))
    cz.cosmica_batch_destroy(b)


def test_autotune_picks_a_valid_shape():
    sets, species, items, b = _setup(cz.PREC_MIXED, counts_seed=2)
    arr = cz.make_items(items)
    tune, rate = cz.cosmica_autotune(b, arr, len(items))
    assert tune.block in (128, 256) and tune.blocks_per_sm >= 1 and rate > 0
    assert tune.compact_period in (0, 64) and tune.queue_order == 1
    cz.cosmica_batch_destroy(b)


@pytest.mark.parametrize("precision", [cz.PREC_MIXED, cz.PREC_MIXED_F64ACC])
def test_launch_shape_compaction_and_queue_order_do_not_change_results(precision):
    """Block size, resident blocks, block compaction and the queue order move particles
    between lanes and change when they start; none may change any exit record."""
    t = torch()
    sets, species, items, b = _setup(precision, counts_seed=3)
    arr = cz.make_items(items)
    total = sum(i[3] for i in items)
    ref = None
    for tune in (cz.cosmica_tuning(128, 0, 0, 0, 0), cz.cosmica_tuning(64, 1, 64, 0, 1),
                 cz.cosmica_tuning(256, 0, 8, 0, 1), cz.cosmica_tuning(32, 2, 1, 0, 0)):
        out = cz.ExitBuffers(total)
        steps = t.zeros(1, dtype=t.int64, device="cuda")
        cz.cosmica_batch_run(b, arr, len(items), out, tuning=tune, steps_out=steps)
        t.cuda.synchronize()
        g = out.numpy()
        assert int(steps.item()) == int(g["steps"].astype(np.int64).sum())
        if ref is None:
            ref = g
        else:
            for k in ref:
                assert np.array_equal(ref[k], g[k]), (tune.block, tune.compact_period, k)
    cz.cosmica_batch_destroy(b)
