"""Multi-rank path on CPU (gloo, world size 2): every rank computes the same
entry partition from the shapes alone (the library's lrb_partition_lpt), the
shards are disjoint and cover the batch, loads are balanced within one entry
of the ideal, each rank's oracle results on its own shard assemble into the
single-process result, each rank's host-only tile list of its share
(lrb_plan_tiles_host) together with the other ranks' covers every output
element of the batch exactly once, and the benchmark's reduction (max of
per-rank times) is what the ranks agree on."""
import heapq
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_07602_gb300 import shard
from paper_2311_07602_gb300 import workloads as W


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        forms, bs, rs = W.variable_shapes(300, seed=17, bmin=16, bmax=256)
        b = W.variable_batch(forms, bs, rs, seed=17)
        owner = shard.lpt_partition(b.m, b.n, b.k, world)
        gathered = [torch.zeros(len(owner), dtype=torch.int32) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(owner))
        same = all(torch.equal(g, gathered[0]) for g in gathered)
        A, B, C = b.A.numpy(), b.B.numpy(), b.C.numpy().copy()
        mine = np.nonzero(owner == rank)[0]
        oracle.gemm_batch([dict(A=A, B=B, C=C, offA=int(b.offA[e]), offB=int(b.offB[e]), offC=int(b.offC[e]),
                                m=int(b.m[e]), n=int(b.n[e]), k=int(b.k[e]), lda=int(b.lda[e]), ldb=int(b.ldb[e]),
                                ldc=int(b.ldc[e])) for e in mine], nthreads=1)
        mask = np.zeros(len(C), dtype=bool)
        for e in mine:
            o = int(b.offC[e])
            mask[o:o + int(b.ldc[e]) * int(b.n[e])] = True
        part = torch.from_numpy(np.where(mask, C, 0.0))
        dist.all_reduce(part)                       # assemble (test-only; the product path never exchanges data)
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        # host-only tiles of this rank's share, entry indices mapped back to
        # the batch's, gathered on every rank
        from paper_2311_07602_gb300 import lrbatch as L
        descs = np.zeros(len(b), dtype=L.DESC_DTYPE)
        descs["A"], descs["B"] = 0x100000, 0x100000
        descs["C"] = 0x1000000000 + 8 * b.offC.astype(np.uint64)
        for key in ("m", "n", "k", "lda", "ldb", "ldc"):
            descs[key] = getattr(b, key)
        tiles = L.lrb_plan_tiles_host(descs[mine], 0).astype(np.int64)
        tiles[:, 0] = mine[tiles[:, 0]]
        counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(counts, torch.tensor([len(tiles)], dtype=torch.int64))
        cap = int(max(c.item() for c in counts))
        padded = torch.full((cap, 5), -1, dtype=torch.int64)
        padded[:len(tiles)] = torch.from_numpy(tiles)
        all_tiles = [torch.zeros((cap, 5), dtype=torch.int64) for _ in range(world)]
        dist.all_gather(all_tiles, padded)
        union = torch.cat([a[a[:, 0] >= 0] for a in all_tiles]).numpy()
        q.put((rank, same, part.numpy() if rank == 0 else None, float(t.item()), union if rank == 0 else None))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_gloo():
    world = 2
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(o[1] for o in out)
    assert all(o[3] == 2.0 for o in out)
    assembled = next(o[2] for o in out if o[0] == 0)
    union = next(o[4] for o in out if o[0] == 0)
    import oracle
    forms, bs, rs = W.variable_shapes(300, seed=17, bmin=16, bmax=256)
    b = W.variable_batch(forms, bs, rs, seed=17)
    A, B, C = b.A.numpy(), b.B.numpy(), b.C.numpy().copy()
    oracle.gemm_batch([dict(A=A, B=B, C=C, offA=int(b.offA[e]), offB=int(b.offB[e]), offC=int(b.offC[e]),
                            m=int(b.m[e]), n=int(b.n[e]), k=int(b.k[e]), lda=int(b.lda[e]), ldb=int(b.ldb[e]),
                            ldc=int(b.ldc[e])) for e in range(len(b))], nthreads=1)
    written = np.zeros(len(C), dtype=bool)
    for e in range(len(b)):
        o = int(b.offC[e])
        written[o:o + int(b.ldc[e]) * int(b.n[e])] = True
    assert np.array_equal(assembled[written], C[written])
    # the ranks' tiles cover every output element of every entry exactly once
    cover = [np.zeros((int(b.m[e]), int(b.n[e])), dtype=np.int32) for e in range(len(b))]
    for e, r0, c0, h, w in union:
        cover[e][r0:r0 + h, c0:c0 + w] += 1
    assert all(np.all(c == 1) for c in cover)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_partition_properties(world):
    forms, bs, rs = W.variable_shapes(2000, seed=4)
    m = bs
    n = np.where(forms == W.FORM_T, rs, bs)
    k = np.where(forms == W.FORM_T, bs, rs)
    owner = shard.lpt_partition(m, n, k, world)
    assert owner.min() >= 0 and owner.max() < world
    loads = shard.shard_loads(m, n, k, owner, world)
    cost = 2.0 * m.astype(float) * n * k
    assert loads.sum() == pytest.approx(cost.sum())
    assert loads.max() - loads.mean() <= cost.max() + 1e-6 * cost.sum()
    assert np.array_equal(owner, shard.lpt_partition(m, n, k, world))


def lpt_reference(cost, world):
    """LPT written out with a heap: entries by decreasing cost (ties: lower
    index), each to the least-loaded rank (ties: lower rank)."""
    order = np.lexsort((np.arange(len(cost)), -np.asarray(cost)))
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(len(cost), dtype=np.int32)
    for e in order:
        load, r = heapq.heappop(heap)
        owner[e] = r
        heapq.heappush(heap, (load + cost[e], r))
    return owner


@pytest.mark.parametrize("world", [1, 2, 5, 8])
def test_library_lpt_matches_heap_statement(world):
    from paper_2311_07602_gb300 import lrbatch as L
    rng = np.random.default_rng(world)
    cost = rng.integers(1, 50, 500).astype(np.float64)          # many ties in cost and in load
    cost[::7] = 0.0
    part, load = L.lrb_partition_lpt(cost, world)
    assert np.array_equal(part, lpt_reference(cost, world))
    assert np.allclose(load, np.bincount(part, weights=cost, minlength=world))
    with pytest.raises(L.LrbError):
        L.lrb_partition_lpt(cost, 0)
    with pytest.raises(L.LrbError):
        L.lrb_partition_lpt(np.array([1.0, -1.0]), 2)
    with pytest.raises(L.LrbError):
        L.lrb_partition_lpt(np.array([1.0, np.nan]), 2)
