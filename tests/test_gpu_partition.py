"""One workload partitioned into shards by ranges of the global particle index
(the multi-GPU path of bench.py, Sec. IV.A), run shard after shard on one GPU
through the C ABI: each shard's exit records equal the single-launch records
of the same particles bit for bit, the shards' histograms -- binned into the
rows of the whole item list via cosmica_work_item.exit_item_plus1 -- sum to the
single-launch histogram exactly, and cosmica_batch_spectrum_hist turns the sum
into the single-launch spectra bit for bit."""
import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from paper_2502_06319_gb300.sharding import items_of, particle_range, partition
from tests.gpu_util import torch

pytestmark = pytest.mark.gpu

NB = 256


@pytest.mark.parametrize("world", [2, 3])
def test_shards_reproduce_the_single_launch(world):
    t = torch()
    jobs = W.config3(n_sets=4, n_e=6, scale=0.01)
    params, species, items = items_of(jobs, 0)
    n_total = sum(i[3] for i in items)
    b = cz.cosmica_batch_create([cz.make_params(p, cz.PREC_MIXED) for p in params],
                                [cz.make_species(s) for s in species])
    bins = cz.make_bins(0.1, 1000.0, NB)
    arr = cz.make_items(items)
    nS = len(items)
    out1 = cz.ExitBuffers(n_total)
    cz.cosmica_batch_run(b, arr, nS, out1)
    J1 = t.empty(nS, dtype=t.float64, device="cuda")
    S1 = t.empty_like(J1)
    H1 = t.empty(nS * (NB + 3), dtype=t.int64, device="cuda")
    cz.cosmica_batch_spectrum(b, arr, nS, out1, bins, J1, S1, H1)
    t.cuda.synchronize()

    Hsum = t.zeros_like(H1)
    for rank in range(world):
        share = partition(items, world, rank)
        pieces, rows = [p for _, p in share], [g for g, _ in share]
        n_r = sum(p[3] for p in pieces)
        lo, hi = particle_range(items, world, rank)
        assert n_r == hi - lo
        o = cz.ExitBuffers(n_r)
        cz.cosmica_batch_run(b, cz.make_items(pieces, rows), len(pieces), o)
        Jr = t.empty_like(J1)
        Sr = t.empty_like(J1)
        Hr = t.empty_like(H1)
        cz.cosmica_batch_spectrum(b, arr, nS, o, bins, Jr, Sr, Hr)
        t.cuda.synchronize()
        for k in ("r", "th", "ph", "lnP", "s", "steps", "status"):
            assert t.equal(getattr(o, k), getattr(out1, k)[lo:hi]), (rank, k)
        # the records carry the global item numbers
        assert t.equal(o.item, out1.item[lo:hi])
        Hsum += Hr
    assert t.equal(Hsum, H1)
    J2 = t.empty_like(J1)
    S2 = t.empty_like(J1)
    cz.cosmica_batch_spectrum_hist(b, arr, nS, bins, Hsum, J2, S2)
    t.cuda.synchronize()
    a, c = J1.cpu().numpy(), J2.cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(c))
    assert np.array_equal(a[~np.isnan(a)], c[~np.isnan(c)])
    s1, s2 = S1.cpu().numpy(), S2.cpu().numpy()
    assert np.array_equal(s1[~np.isnan(s1)], s2[~np.isnan(s2)])
    cz.cosmica_batch_destroy(b)


def test_spectrum_hist_rejects_host_memory():
    t = torch()
    b = cz.cosmica_batch_create([cz.make_params(W.params(), cz.PREC_MIXED)], [cz.make_species(W.PROTON)])
    arr = cz.make_items([(0, 0, 1.0, 4, 0, 1)])
    H = t.zeros(NB + 3, dtype=t.int64)
    J = t.empty(1, dtype=t.float64, device="cuda")
    with pytest.raises(cz.CosmicaError):
        cz.cosmica_batch_spectrum_hist(b, arr, 1, cz.make_bins(0.1, 1000.0, NB), H, J, J)
    cz.cosmica_batch_destroy(b)
