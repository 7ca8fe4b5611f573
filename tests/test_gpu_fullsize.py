"""Config 3 at its full size (7.4e7 quasi-particles, 64 heliospheres x 3 species
x 30 energies) in the launch configuration bench.py times: the autotuned shape,
one persistent launch, graph replay.  Mixed paths are chaotic at the rounding
level, so the oracle cannot follow them one by one; what holds at any size is
checked instead:
  * every path exits (no step limit, no non-finite state) and every exit record
    names a valid work item; the histograms count every particle;
  * sampled items, re-run alone, give bit-identical exit records (a path
    depends only on its seed, identity, parameters, species and energy);
  * the spectrum of the smallest item of each species agrees with the FP64
    oracle's within 3 sigma (the oracle runs the same particles);
  * the twelve items of the stored oracle result (tests/golden/oracle_c3_items.json:
    both polarity epochs, tilts 73/64/11/8 deg, p/He-4/e-, 4-5e4 paths each), taken
    from this full-size launch, agree with it within 3 sigma and 0.5 %.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from paper_2502_06319_gb300.sharding import items_of
from tests.gpu_util import torch

pytestmark = pytest.mark.gpu


def test_config3_full_size_properties(orc):
    t = torch()
    jobs = W.config3()
    params, species, items = items_of(jobs, 0)
    n_total = sum(i[3] for i in items)
    assert n_total > 7e7
    b = cz.cosmica_batch_create([cz.make_params(p, cz.PREC_MIXED) for p in params],
                                [cz.make_species(s) for s in species])
    arr = cz.make_items(items)
    tune, _ = cz.cosmica_autotune(b, arr, len(items))
    tune.use_graph = 1
    s = t.cuda.Stream()
    out = cz.ExitBuffers(n_total)
    steps = t.zeros(1, dtype=t.int64, device="cuda")
    with t.cuda.stream(s):
        cz.cosmica_batch_run(b, arr, len(items), out, tuning=tune, steps_out=steps, stream=s)
    s.synchronize()
    status = out.status
    assert bool((status == cz.PATH_EXIT).all())
    item = out.item.to(t.int64)
    assert int(item.min()) >= 0 and int(item.max()) < len(items)
    nb = 512
    J = t.empty(len(items), dtype=t.float64, device="cuda")
    S = t.empty_like(J)
    H = t.empty(len(items) * (nb + 3), dtype=t.int64, device="cuda")
    cz.cosmica_batch_spectrum(b, arr, len(items), out, cz.make_bins(0.1, 1000.0, nb), J, S, H)
    t.cuda.synchronize()
    Hn = H.cpu().numpy().reshape(len(items), nb + 3)
    counts = np.array([i[3] for i in items])
    assert np.array_equal(Hn.sum(axis=1), counts)
    assert int(steps.item()) == int(out.steps.to(t.int64).sum().item())

    # sampled items alone, bit for bit
    prefix = np.concatenate([[0], np.cumsum(counts)])
    rng = np.random.default_rng(3)
    pick = rng.choice(len(items), 3, replace=False)
    for k in pick:
        pi, si, T_, n, fp, sd = items[k]
        one = cz.cosmica_batch_create([cz.make_params(params[pi], cz.PREC_MIXED)],
                                      [cz.make_species(species[si])])
        o1 = cz.ExitBuffers(n)
        cz.cosmica_batch_run(one, cz.make_items([(0, 0, T_, n, fp, sd)]), 1, o1)
        t.cuda.synchronize()
        alone = o1.numpy()
        cz.cosmica_batch_destroy(one)
        lo, hi = prefix[k], prefix[k + 1]
        for key in ("r", "th", "ph", "lnP", "s"):
            assert t.equal(getattr(out, key)[lo:hi].cpu(), t.as_tensor(alone[key])), (k, key)
        assert np.array_equal(out.steps[lo:hi].cpu().numpy().view(np.uint32), alone["steps"])

    # the spectra of the smallest item of each species against the FP64 oracle (same particles)
    Jn, Sn = J.cpu().numpy(), S.cpu().numpy()
    for si_want in range(len(species)):
        cand = [j for j, it in enumerate(items) if it[1] == si_want]
        k = min(cand, key=lambda j: items[j][3])
        pi, si, T_, n, fp, sd = items[k]
        o = orc.run(params[pi], species[si], [T_], [n], seed=sd, first_pid=fp)
        Ho = orc.histogram(o, 1, 0.1, 1000.0, nb)
        Jo, So = orc.spectrum_from_hist(Ho, species[si], [T_], 0.1, 1000.0, nb)
        print(f"full-size item {k} ({species[si]}, T {T_:.3g}, n {n}): mixed/oracle - 1 = {Jn[k] / Jo[0] - 1:.4f}, "
              f"sigma_rel {So[0] / Jo[0]:.4f}")
        assert abs(Jn[k] - Jo[0]) <= 3 * np.hypot(Sn[k], So[0]), (k, Jn[k], Jo[0], Sn[k], So[0])

    # the stored oracle items, from the full-size launch
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_c3_items.json")) as f:
        golden = json.load(f)
    for rec in golden["items"]:
        k = rec["item"]
        assert (items[k][3], items[k][4]) == (rec["n"], rec["first_pid"])
        d = Jn[k] - rec["J"]
        assert abs(d) <= 3.0 * math.hypot(Sn[k], rec["sigma"]) and abs(d) <= 0.005 * rec["J"], (k, d / rec["J"])
    cz.cosmica_batch_destroy(b)
