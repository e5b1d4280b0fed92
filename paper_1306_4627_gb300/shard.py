"""Partition of a batch of independent pairs over ranks (one rank per GPU): no data moves between ranks.

Pairs are independent problems, so the batch shards by pair. The split balances cells (m * n, the work of a pair):
pairs are taken largest first and each goes to the rank with the fewest cells so far (ties to the lower rank), a
deterministic greedy rule that every rank evaluates for itself, so the ranks agree without communicating.
"""

from __future__ import annotations

import heapq

import numpy as np


def partition_pairs(m, n, world: int) -> list[np.ndarray]:
    """Indices of the pairs of each rank (ascending within a rank) for pair lengths m[k], n[k]."""
    if world < 1:
        raise ValueError("world must be at least 1")
    m = np.asarray(m, dtype=np.int64)
    n = np.asarray(n, dtype=np.int64)
    if m.shape != n.shape:
        raise ValueError("m and n must have the same length")
    cells = m * n
    order = np.lexsort((np.arange(len(cells)), -cells))  # largest first, then by index
    heap = [(0, r) for r in range(world)]
    owner = np.empty(len(cells), dtype=np.int64)
    for k in order:
        load, r = heapq.heappop(heap)
        owner[k] = r
        heapq.heappush(heap, (load + int(cells[k]), r))
    return [np.flatnonzero(owner == r) for r in range(world)]


def shard_cells(m, n, parts) -> list[int]:
    """Cells of each rank's shard."""
    m = np.asarray(m, dtype=np.int64)
    n = np.asarray(n, dtype=np.int64)
    return [int((m[p] * n[p]).sum()) for p in parts]
