"""Multi-rank path on CPU (gloo, world size 2): every rank computes the same
entry partition from the shapes alone, the shards are disjoint and cover the
batch, loads are balanced within one entry of the ideal, each rank's oracle
results on its own shard assemble into the single-process result, and the
benchmark's reduction (max of per-rank times) is what the ranks agree on."""
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
        q.put((rank, same, part.numpy() if rank == 0 else None, float(t.item())))
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
