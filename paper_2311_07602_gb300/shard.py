"""Entry sharding across GPUs (one process per GPU, no data-path collective).

Batch entries are independent (the paper's batch loop, Alg. 2 loop 1, has no
cross-entry dependence), so a multi-GPU run partitions the entries: longest
processing time first over the per-entry cost 2 m n k, each entry to the
currently least-loaded rank (the library's lrb_partition_lpt).  Every rank
computes the same partition from the shapes alone, so no exchange is needed;
each rank then plans and runs its own entries on its own GPU, and results
stay where their C lives.  In one process that drives several GPUs,
lrbatch.MultiPlan (lrb_multi_plan_create) does the same over several handles.
"""
from __future__ import annotations

import numpy as np

from . import lrbatch as L


def entry_costs(m, n, k) -> np.ndarray:
    return 2.0 * np.asarray(m, dtype=np.float64) * np.asarray(n, dtype=np.float64) * np.asarray(k, dtype=np.float64)


def lpt_partition(m, n, k, world: int) -> np.ndarray:
    """Rank of every entry (int32 array): LPT over cost 2 m n k, ties by entry index."""
    part, _ = L.lrb_partition_lpt(entry_costs(m, n, k), world)
    return part


def shard_loads(m, n, k, owner: np.ndarray, world: int) -> np.ndarray:
    return np.bincount(owner, weights=entry_costs(m, n, k), minlength=world)
