"""Sharding of the batched form over GPUs (one process per GPU, no collective).

Independent systems are dealt to ranks by greedy longest-processing-time (LPT) order
on an estimated cost, each rank runs its share through the batched C ABI calls on its
own GPU, and the per-system results are gathered on the host of rank 0 (an
object gather over torch.distributed, outside the data path).  A single system is not
sharded: its factorization would need separator exchanges at every tree level and its
block GCR an allreduce of the Gram matrices per iteration.
"""
from __future__ import annotations

import heapq


def estimated_cost(L: int, dim: int = 2) -> float:
    """Nested-dissection work estimate of one system: L^1.5 in 2D, L^2 in 3D."""
    return float(L) ** (1.5 if dim == 2 else 2.0)


def lpt_partition(costs, n_ranks: int):
    """Greedy LPT: systems in decreasing cost order, each to the least-loaded rank.

    Returns one list of system indices per rank (ascending within a rank); ties of load
    go to the smaller rank, ties of cost to the smaller index, so every rank computes
    the same partition."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(n_ranks)]
    heapq.heapify(heap)
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def run_sharded(n_systems: int, costs, run_share, rank: int, world: int, group=None):
    """Run `run_share(indices) -> {index: result}` on this rank's share and gather all
    results on rank 0 (returned there as a list in system order; None elsewhere)."""
    parts = lpt_partition(costs, world)
    mine = run_share(parts[rank]) if parts[rank] else {}
    if world == 1:
        return [mine[i] for i in range(n_systems)]
    import torch.distributed as dist
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(mine, gathered, dst=0, group=group)
    if rank != 0:
        return None
    out = {}
    for d in gathered:
        out.update(d)
    return [out[i] for i in range(n_systems)]
