"""Entry sharding across GPUs (one process per GPU, no data-path collective).

Batch entries are independent (the paper's batch loop, Alg. 2 loop 1, has no
cross-entry dependence), so a multi-GPU run partitions the entries: longest
processing time first over the per-entry cost 2 m n k, each entry to the
currently least-loaded rank.  Every rank computes the same partition from
the shapes alone, so no exchange is needed; each rank then plans and runs
its own entries on its own GPU, and results stay where their C lives.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(m, n, k, world: int) -> np.ndarray:
    """Rank of every entry (int32 array): LPT over cost 2 m n k, ties by entry index."""
    cost = 2.0 * np.asarray(m, dtype=np.float64) * np.asarray(n, dtype=np.float64) * np.asarray(k, dtype=np.float64)
    order = np.lexsort((np.arange(len(cost)), -cost))
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(len(cost), dtype=np.int32)
    for e in order:
        load, r = heapq.heappop(heap)
        owner[e] = r
        heapq.heappush(heap, (load + cost[e], r))
    return owner


def shard_loads(m, n, k, owner: np.ndarray, world: int) -> np.ndarray:
    cost = 2.0 * np.asarray(m, dtype=np.float64) * np.asarray(n, dtype=np.float64) * np.asarray(k, dtype=np.float64)
    return np.bincount(owner, weights=cost, minlength=world)
