"""Multi-GPU host logic of the batched path (weak scaling).

Quasi-particles are independent (Sec. IV.A), so N GPUs need no exchange on the
data path: rank k propagates its own copy of the workload with particle
identities offset by k * 2^40 and seeds offset by k, and the only collectives
are the barrier around the timed region and the reduction of the timing
(max over ranks) and of the step counts (sum over ranks).
"""
from __future__ import annotations

PID_STRIDE = 1 << 40


def items_of(jobs, rank: int):
    """Work items (param_idx, species_idx, T, n, first_pid, seed) of all jobs for `rank`,
    with de-duplicated parameter sets and species."""
    params, pkeys, species, skeys, items = [], {}, [], {}, []
    pid = 0
    base = rank * PID_STRIDE
    for j in jobs:
        pk = tuple(sorted(j.params.items()))
        if pk not in pkeys:
            pkeys[pk] = len(params)
            params.append(j.params)
        sk = tuple(sorted(j.species.items()))
        if sk not in skeys:
            skeys[sk] = len(species)
            species.append(j.species)
        for T, n in zip(j.T_in, j.n_per_energy):
            items.append((pkeys[pk], skeys[sk], T, n, base + pid, j.seed + 7919 * rank))
            pid += n
    if pid >= PID_STRIDE:
        raise ValueError("workload exceeds the per-rank particle-identity range")
    return params, species, items


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
