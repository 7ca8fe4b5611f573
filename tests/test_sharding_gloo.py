"""Multi-GPU host logic on CPU, with two gloo ranks: the partition of one
workload by contiguous ranges of the global particle index (the paper's
distribution of the energy bins over GPUs, Sec. IV.A) and the merge of the
per-rank histograms by one all-reduce.  The ranks run the FP64 oracle on
their shares (the merge is the same integer sum whatever computed the
histograms); the merged histogram must equal the single-rank one bit for bit.
The replica mode (weak scaling) and the timing reduction are checked too."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2502_06319_gb300 import workloads as W
from paper_2502_06319_gb300.sharding import (PID_STRIDE, items_of, merge_histograms, particle_range, partition,
                                             reduce_timing)

NB = 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _small_workload():
    """Two heliospheres x 3 species x 5 energies of the batched workload's ranges, 1-40
    particles per item, at energies where paths are short (the oracle finishes in seconds)."""
    jobs = W.config3(n_sets=2, n_e=5, n_lo=1, n_hi=40)
    for j in jobs:
        j.T_in = [5.0, 10.0, 20.0, 40.0, 80.0]
    return jobs


def _oracle_hist(params, species, pieces, rows, n_rows, threads):
    """Histogram (rows x (NB + 3)) of the oracle's exit records of the given item pieces,
    each binned into the row of its global item."""
    from oracle import oracle as O
    prm, spc, T, pid, seed, row = [], [], [], [], [], []
    for (pi, si, T_, n, fp, sd), r in zip(pieces, rows):
        prm += [pi] * n
        spc += [si] * n
        T += [T_] * n
        pid += range(fp, fp + n)
        seed += [sd] * n
        row += [r] * n
    out = O.run_particles(params, species, np.array(prm, np.uint32), np.array(spc, np.uint32),
                          np.array(T, np.float64), np.array(pid, np.uint64), np.array(seed, np.uint64),
                          threads=threads)
    out["energy"] = np.array(row, np.int64)
    return O.histogram(out, n_rows, 0.1, 1000.0, NB).astype(np.int64)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    params, species, items = items_of(_small_workload(), 0)
    share = partition(items, world, rank)
    H = torch.from_numpy(_oracle_hist(params, species, [p for _, p in share], [g for g, _ in share],
                                      len(items), threads=2))
    merge_histograms(dist, H)
    # replicas: every rank holds the whole workload with its own identities
    _, _, rep = items_of(_small_workload(), rank)
    ms, steps = reduce_timing(dist, 100.0 + 50.0 * rank, 1000 * (rank + 1))
    q.put((rank, share, H.numpy(), [(it[4], it[4] + it[3]) for it in rep], [it[5] for it in rep], ms, steps))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_tiles_the_item_list():
    _, _, items = items_of(_small_workload(), 0)
    total = sum(it[3] for it in items)
    for world in (1, 2, 3, 7):
        covered = {}
        for rank in range(world):
            lo, hi = particle_range(items, world, rank)
            n_rank = 0
            for g, (pi, si, T, n, fp, sd) in partition(items, world, rank):
                assert (pi, si, T, sd) == (items[g][0], items[g][1], items[g][2], items[g][5])
                assert n >= 1
                covered.setdefault(g, []).append((fp, fp + n))
                n_rank += n
            assert n_rank == hi - lo
        for g, it in enumerate(items):
            runs = sorted(covered.get(g, []))
            if it[3] == 0:
                assert not runs
                continue
            # the pieces of an item are contiguous, disjoint and cover its identities exactly
            assert runs[0][0] == it[4] and runs[-1][1] == it[4] + it[3]
            assert all(a[1] == b[0] for a, b in zip(runs, runs[1:]))
        assert sum(it[3] for it in items) == total
    with pytest.raises(ValueError):
        particle_range(items, 2, 2)


def test_two_ranks_merged_histogram_equals_one_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    params, species, items = items_of(_small_workload(), 0)
    H1 = _oracle_hist(params, species, items, list(range(len(items))), len(items), threads=0)
    (_, share0, Hm0, rep0, seeds0, ms0, st0), (_, share1, Hm1, rep1, seeds1, ms1, st1) = res
    # each rank took a non-empty share and the shares split at least one item between them
    assert share0 and share1
    assert np.array_equal(Hm0, Hm1)
    assert np.array_equal(Hm0, H1), "merged two-rank histogram differs from the single-rank one"
    assert int(H1.sum()) == sum(it[3] for it in items)
    # replicas: disjoint identities and seeds on every rank
    assert all(b <= PID_STRIDE for _, b in rep0) and all(a >= PID_STRIDE for a, _ in rep1)
    assert set(seeds0).isdisjoint(seeds1)
    # max over ranks of the time, sum of the steps, identical on every rank
    assert ms0 == ms1 == 150.0 and st0 == st1 == 3000.0


def test_single_rank_passthrough():
    assert reduce_timing(None, 12.5, 7) == (12.5, 7)
    merge_histograms(None, torch.zeros(3))
    with pytest.raises(ValueError):
        items_of([W.Job(W.params(), W.PROTON, [1.0], [PID_STRIDE], seed=1)], 0)


def test_pieces_carry_their_global_rows_into_the_work_items():
    # what bench.py hands to cosmica_batch_run on each rank: the pieces' work items carry
    # exit_item_plus1 = global row + 1 (the histogram row of the whole item list), their own
    # particle count and first identity; an unsharded list carries 0 (its own numbering)
    from paper_2502_06319_gb300 import cosmica as cz
    _, _, items = items_of(_small_workload(), 0)
    for world in (2, 3):
        for rank in range(world):
            share = partition(items, world, rank)
            arr = cz.make_items([p for _, p in share], [g for g, _ in share])
            for k, (g, p) in enumerate(share):
                w = arr[k]
                assert w.exit_item_plus1 == g + 1 and w.n == p[3] and w.first_pid == p[4]
                assert (w.param_idx, w.species_idx, w.T_GeVn, w.seed) == (items[g][0], items[g][1],
                                                                           items[g][2], items[g][5])
    arr = cz.make_items(items)
    assert all(arr[k].exit_item_plus1 == 0 for k in range(len(items)))
