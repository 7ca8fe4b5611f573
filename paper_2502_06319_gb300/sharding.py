"""Multi-GPU host logic of the batched path.

Quasi-particles are independent and the only quantity the GPUs exchange is
the integer exit histogram (the paper distributes the energy bins over the
GPUs and collects their histograms, Sec. IV.A).  Two ways to use N GPUs:

  * partition (strong scaling, the default of bench.py): one workload is cut
    into N contiguous ranges of the global particle index (the prefix sum of
    the items' counts); rank k propagates particles
    floor(k T / N) <= g < floor((k+1) T / N), T the total.  An item that
    straddles a cut is split; its pieces keep the item's first particle
    identity plus their offset, so every path is the one a single GPU would
    run.  Each rank bins its exit records into the rows of the GLOBAL item list
    (the pieces carry their global item number into the exit records) and one
    all-reduce of the u64 histograms gives every rank the 1-GPU histogram,
    from which the spectra follow.  Integer sums are exact and
    order-independent, so the merged histogram equals the 1-GPU one bit for bit.
  * replicas (weak scaling): rank k propagates its own copy of the workload
    with particle identities offset by k * 2^40 and seeds offset by k; no
    exchange at all.
"""
from __future__ import annotations

# the work-item list of a set of jobs is input description, kept with the input generators
from .workloads import PID_STRIDE, items_of  # noqa: E402,F401


def particle_range(items, world: int, rank: int):
    """[lo, hi) of the global particle index that `rank` of `world` propagates."""
    if not (world >= 1 and 0 <= rank < world):
        raise ValueError(f"rank {rank} of world {world}")
    total = sum(int(it[3]) for it in items)
    return rank * total // world, (rank + 1) * total // world


def partition(items, world: int, rank: int):
    """This rank's share of the work items: a list of (global item index, piece), the
    piece an item tuple (param_idx, species_idx, T, n, first_pid, seed) covering the
    part of the global item that falls in the rank's particle range.  Pieces keep
    the global particle identities (first_pid + offset within the item)."""
    lo, hi = particle_range(items, world, rank)
    out = []
    start = 0
    for i, it in enumerate(items):
        pi, si, T, n, fp, sd = it[:6]
        a, b = max(lo, start), min(hi, start + int(n))
        if a < b:
            out.append((i, (pi, si, T, b - a, fp + (a - start), sd)))
        start += int(n)
    return out


def merge_histograms(dist, hist) -> None:
    """Sum the per-rank histograms of the global item list in place (one all-reduce:
    NCCL on GPUs, gloo in the CPU tests).  No-op without a process group."""
    if dist is None:
        return
    dist.all_reduce(hist, op=dist.ReduceOp.SUM)


def reduce_timing(dist, total_ms: float, steps: float, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the steps)."""
    import torch
    if dist is None:
        return total_ms, steps
    t = torch.tensor([total_ms, float(steps)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])
