"""Multi-GPU host logic on CPU: two gloo ranks build their shards of a
workload and reduce the timing exactly as bench.py does on N GPUs."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2502_06319_gb300 import workloads as W
from paper_2502_06319_gb300.sharding import PID_STRIDE, items_of, reduce_timing


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = W.config3(n_sets=3, scale=0.01)
    params, species, items = items_of(jobs, rank)
    ms, steps = reduce_timing(dist, 100.0 + 50.0 * rank, 1000 * (rank + 1))
    pids = [(it[4], it[4] + it[3]) for it in items]
    q.put((rank, len(params), len(species), pids, [it[5] for it in items], ms, steps))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_shards_and_reductions():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, np0, ns0, pids0, seeds0, ms0, st0), (r1, np1, ns1, pids1, seeds1, ms1, st1) = res
    assert (np0, ns0) == (np1, ns1) == (3, 3)
    # each rank holds the whole workload with its own identities: weak scaling
    assert len(pids0) == len(pids1) == 3 * 3 * 30
    assert all(a[1] <= PID_STRIDE for a in pids0) and all(b[0] >= PID_STRIDE for b in pids1)
    flat = sorted(pids0 + pids1)
    assert all(flat[i][1] <= flat[i + 1][0] for i in range(len(flat) - 1))   # no shared particle
    assert set(seeds0).isdisjoint(seeds1)
    # max over ranks of the time, sum of the steps, identical on every rank
    assert ms0 == ms1 == 150.0 and st0 == st1 == 3000.0


def test_single_rank_passthrough():
    assert reduce_timing(None, 12.5, 7) == (12.5, 7)
    with pytest.raises(ValueError):
        items_of([W.Job(W.params(), W.PROTON, [1.0], [PID_STRIDE], seed=1)], 0)
