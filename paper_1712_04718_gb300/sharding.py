"""Sharding an ensemble of independent systems over ranks (host logic only).

A single system is not sharded: one GB300 holds the largest workload many
times over, so N ranks run N replicas.  An ensemble of independent systems
(the batched form, se_batch_*) shards naturally: each rank evaluates its own
subset of the systems and no data crosses ranks; only the timing is reduced
(the slowest rank's time).  Every rank computes the same assignment from the
same inputs, so no exchange is needed to agree on it.
"""
import math


def system_cost(N, M, P):
    """Work of one system's evaluation: N P^3 for the spread and the gather
    plus M^3 log2 M for the transforms."""
    return float(N) * P ** 3 + float(M) ** 3 * math.log2(max(M, 2))


def partition_systems(costs, ws):
    """Systems -> ranks, balanced by cost: largest first onto the least
    loaded rank (ties to the lower rank).  Returns the sorted system indices
    of each of the ws ranks (a rank may get none when ws > len(costs))."""
    load = [0.0] * ws
    parts = [[] for _ in range(ws)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(ws), key=lambda r: (load[r], r))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def shard(Ns, Ms, P, ws, rank):
    """Indices of the systems rank `rank` of ws evaluates (Ns atoms and Ms
    grid points per dimension per system, support P)."""
    return partition_systems([system_cost(n, m, P) for n, m in zip(Ns, Ms)], ws)[rank]


def max_over_ranks(value, ws, device):
    """The largest value over all ranks (the slowest rank's time); `value`
    itself when ws == 1.  Needs an initialised torch.distributed group."""
    if ws <= 1:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.item()
