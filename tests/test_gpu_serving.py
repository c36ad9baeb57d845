"""The serving queue (continuous batching) through the C ABI.

* Each request's result is bitwise the same alone (one request at a time)
  and in a mix (all submitted together, admitted in overlapping waves), and
  matches the oracle within the FP64 tolerance.
* Admission never reserves more than the HBM budget; a request larger than
  the budget is refused (LRB_ERR_BUDGET); a full waiting FIFO refuses with
  LRB_ERR_QUEUE_FULL; waits are bounded (LRB_ERR_TIMEOUT).
"""
import numpy as np
import pytest
import torch

from paper_2311_07602_gb300 import lrbatch as L
from paper_2311_07602_gb300 import workloads as W
from tests.parity import check_entries, host, oracle_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    h = L.Handle(0)
    yield h
    h.close()


def requests(nreq, seed, max_products=12, bmax=300):
    """One variable batch; request q owns a contiguous slice of its entries."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(1, max_products + 1, nreq)
    forms, bs, rs = W.variable_shapes(int(counts.sum()), seed=seed, bmin=16, bmax=bmax, ranks=(8, 16, 32, 64))
    batch = W.variable_batch(forms, bs, rs, seed=seed)
    bounds = np.concatenate([[0], np.cumsum(counts)])
    return batch, [(int(bounds[q]), int(bounds[q + 1])) for q in range(nreq)]


def test_alone_equals_mix_bitwise(handle):
    batch, reqs = requests(16, seed=51)
    Ah, Bh, C0 = host(batch.A), host(batch.B), host(batch.C)
    # alone: one request in flight at a time
    dev1 = batch.to("cuda")
    d1 = L.descs_for(dev1)
    with L.Queue(handle, budget_bytes=40 << 30, max_inflight=1) as q:
        for lo, hi in reqs:
            st, t = q.submit(d1[lo:hi])
            assert st == L.LRB_OK
            assert q.wait(t, 60000) == L.LRB_OK
    alone = host(dev1.C)
    # mix: everything submitted at once, several waves overlapping
    dev2 = batch.to("cuda")
    d2 = L.descs_for(dev2)
    with L.Queue(handle, budget_bytes=40 << 30, max_inflight=4) as q:
        q.set_limits(4096, max_wave_entries=24)   # force several waves
        tickets = []
        for lo, hi in reqs:
            st, t = q.submit(d2[lo:hi])
            assert st == L.LRB_OK
            tickets.append(t)
        for t in tickets:
            assert q.wait(t, 60000) == L.LRB_OK
        s = q.stats()
        assert s["completed"] == len(reqs) and s["waves"] >= 2
        assert s["p99_ms"] >= s["p50_ms"] > 0
    mix = host(dev2.C)
    assert np.array_equal(alone.view(np.uint64), mix.view(np.uint64))
    exp = oracle_batch(Ah, Bh, C0, batch)
    check_entries(mix, exp, Ah, Bh, C0, batch)


def test_budget_is_respected(handle):
    batch, reqs = requests(24, seed=52, max_products=6, bmax=500)
    dev = batch.to("cuda")
    d = L.descs_for(dev)
    sizes = [int(np.sum(8 * (batch.m[lo:hi].astype(np.int64) * batch.k[lo:hi] + batch.k[lo:hi] * batch.n[lo:hi] +
                             batch.m[lo:hi] * batch.n[lo:hi]) + 64 * (hi - lo))) for lo, hi in reqs]
    budget = 3 * max(sizes)
    with L.Queue(handle, budget_bytes=budget, max_inflight=4) as q:
        tickets = []
        for lo, hi in reqs:
            st, t = q.submit(d[lo:hi])
            assert st == L.LRB_OK
            tickets.append(t)
        for t in tickets:
            assert q.wait(t, 60000) == L.LRB_OK
        s = q.stats()
        assert 0 < s["peak_reserved_bytes"] <= budget
        assert s["reserved_bytes"] == 0 and s["completed"] == len(reqs)
    # a request larger than the whole budget is refused
    with L.Queue(handle, budget_bytes=min(sizes) - 1, max_inflight=1) as q:
        lo, hi = reqs[int(np.argmin(sizes))]
        st, _ = q.submit(d[lo:hi])
        assert st == L.LRB_ERR_BUDGET
        assert q.stats()["rejected_budget"] == 1


def test_queue_full_and_bounded_waits(handle):
    # one long request occupies the whole budget; tiny ones queue behind it
    big = W.uniform_batch(W.FORM_O, 2048, 128, 6, seed=9, device="cuda")
    dbig = L.descs_for(big)
    big_bytes = int(np.sum(8 * (big.m.astype(np.int64) * big.k + big.k * big.n + big.m * big.n) + 64))
    tiny = W.uniform_batch(W.FORM_T, 16, 8, 64, seed=10, device="cuda")
    dt = L.descs_for(tiny)
    with L.Queue(handle, budget_bytes=big_bytes, max_inflight=2) as q:
        q.set_limits(max_waiting=8)
        st, tb = q.submit(dbig)
        assert st == L.LRB_OK
        got = [q.submit(dt[i:i + 1])[0] for i in range(40)]
        assert got.count(L.LRB_ERR_QUEUE_FULL) >= 40 - 9
        assert q.wait(tb, 0) in (L.LRB_ERR_TIMEOUT, L.LRB_OK)
        assert q.poll(tb) in (L.LRB_ERR_TIMEOUT, L.LRB_OK)
        assert q.wait(tb, 60000) == L.LRB_OK
        assert q.poll(tb) == L.LRB_OK
        assert q.latency(tb) > 0
        assert q.poll(123456789) == L.LRB_ERR_INVALID
    del big, tiny


def test_split_precision_waves_alone_equals_mix(handle):
    """Waves in BF16 S=3 split precision: each request's result is bitwise the
    same alone and in a mix, and matches the split oracle within the binary64
    regrouping bound."""
    import oracle
    from oracle import PRESETS
    from tests.parity import entry_view
    batch, reqs = requests(10, seed=53, max_products=5, bmax=400)
    Ah, Bh, C0 = host(batch.A), host(batch.B), host(batch.C)
    outs = []
    for slots, wave_entries in ((1, 1 << 16), (4, 6)):
        dev = batch.to("cuda")
        d = L.descs_for(dev)
        with L.Queue(handle, budget_bytes=40 << 30, max_inflight=slots) as q:
            q.set_precision(L.LRB_PREC_SPLIT_BF16_S3)
            q.set_limits(4096, max_wave_entries=wave_entries)
            tickets = []
            for lo, hi in reqs:
                st, t = q.submit(d[lo:hi])
                assert st == L.LRB_OK
                tickets.append(t)
                if slots == 1:
                    assert q.wait(t, 60000) == L.LRB_OK
            for t in tickets:
                assert q.wait(t, 60000) == L.LRB_OK
        outs.append(host(dev.C))
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
    p = PRESETS["bf16_s3"]
    for e in range(len(batch)):
        m, n, k = int(batch.m[e]), int(batch.n[e]), int(batch.k[e])
        A = entry_view(Ah, int(batch.offA[e]), m, k, int(batch.lda[e])).copy()
        B = entry_view(Bh, int(batch.offB[e]), k, n, int(batch.ldb[e])).copy()
        C = entry_view(C0, int(batch.offC[e]), m, n, int(batch.ldc[e])).copy()
        exp = oracle.split_gemm(A, B, C, p)
        got = entry_view(outs[1], int(batch.offC[e]), m, n, int(batch.ldc[e]))
        nadd = ((k + p.kc - 1) // p.kc) * (len(p.levels()) + 1)
        assert np.all(np.abs(got - exp) <= 2 * oracle.gamma(nadd) * oracle.recombination_magnitude(A, B, C, p))
