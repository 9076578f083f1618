"""Instance sharding over GPUs (one process per GPU).

Every TDSE instance is independent, so a multi-GPU run is a partition of the instance list with no
collective on the data path; torch.distributed is only used for the timing barrier and the
max-over-ranks of the measured time.  Uniform batches take contiguous blocks; uneven batches are
balanced by the cost N x Nt of each instance with the longest-processing-time-first rule (sort by
cost, give each instance to the least loaded rank), which keeps the largest rank load within 4/3 of
the optimum.
"""
from __future__ import annotations

import heapq

import numpy as np


def contiguous(n: int, world: int, rank: int) -> slice:
    """Rank `rank`'s block of n instances split into `world` nearly equal contiguous blocks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return slice(lo, lo + base + (1 if rank < extra else 0))


def lpt(costs, world: int):
    """Index arrays (one per rank, each sorted) balancing sum(costs) over `world` ranks."""
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def instance_cost(N, n_steps):
    """Work of an instance in grid-point steps."""
    return np.asarray(N, dtype=np.float64) * np.asarray(n_steps, dtype=np.float64)
