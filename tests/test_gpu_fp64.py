"""GPU parity of the FP64 path against the oracle, through the C ABI.

Tolerance: relative Frobenius error <= 1e-13 per entry, and every element
within 2 gamma_{k+1} (|C0| + |A||B|) of the oracle (both results are within
gamma_{k+1} of the exact value for any summation order).  Integer-valued,
identity and permutation inputs are exact in any order, so there the check
is bitwise.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2311_07602_gb300 import lrbatch as L
from paper_2311_07602_gb300 import workloads as W
from tests.parity import (c0_at, check_entries, draw_samples, entry_view, host, oracle_batch,
                          sample_check)

pytestmark = pytest.mark.gpu

NAN_CANARY = np.frombuffer(np.uint64(0x7FF8DEADBEEF0001).tobytes(), dtype=np.float64)[0]


@pytest.fixture(scope="module")
def handle():
    h = L.Handle(0)
    yield h
    h.close()


def ragged_batch(shapes, pad, seed, dist="normal", guard=64):
    """Entries with ld = rows + pad, separated by `guard` canary elements;
    the ld padding rows are canaries too."""
    rng = np.random.default_rng(seed)
    offs = {"A": [], "B": [], "C": []}
    tot = {"A": guard, "B": guard, "C": guard}
    m_, n_, k_, la, lb, lc = [], [], [], [], [], []
    for (m, n, k) in shapes:
        lda, ldb, ldc = m + pad, k + pad, m + pad
        for key, size in (("A", lda * k), ("B", ldb * n), ("C", ldc * n)):
            offs[key].append(tot[key])
            tot[key] += size + guard
        m_.append(m), n_.append(n), k_.append(k), la.append(lda), lb.append(ldb), lc.append(ldc)
    bufs = {}
    for key in "ABC":
        x = np.full(tot[key], NAN_CANARY)
        bufs[key] = x
    for e, (m, n, k) in enumerate(shapes):
        for key, rows, cols, ld in (("A", m, k, la[e]), ("B", k, n, lb[e]), ("C", m, n, lc[e])):
            v = entry_view(bufs[key], offs[key][e], rows, cols, ld)
            if dist == "int":
                v[...] = rng.integers(-8, 9, (rows, cols))
            else:
                v[...] = rng.standard_normal((rows, cols))
    arr = lambda x: np.asarray(x, dtype=np.int32)
    return W.Batch(torch.from_numpy(bufs["A"]), torch.from_numpy(bufs["B"]), torch.from_numpy(bufs["C"]),
                   arr(m_), arr(n_), arr(k_), arr(la), arr(lb), arr(lc),
                   np.asarray(offs["A"], dtype=np.int64), np.asarray(offs["B"], dtype=np.int64),
                   np.asarray(offs["C"], dtype=np.int64))


RAGGED = [(1, 1, 1), (37, 5, 19), (100, 70, 33), (64, 8, 16), (129, 65, 130), (33, 129, 3), (200, 16, 200),
          (65, 64, 17), (31, 31, 64), (256, 16, 256)]


def run_gpu(handle, batch_host, launch="persistent", **opts):
    dev = batch_host.to("cuda")
    plan = handle.plan(L.descs_for(dev), **opts)
    if launch == "plain":
        plan.launch_plain()
    else:
        plan.launch()
    torch.cuda.synchronize()
    plan.close()
    return host(dev.C)


@pytest.mark.parametrize("variant", range(10))
def test_every_variant_ragged_with_canaries(handle, variant):
    b = ragged_batch(RAGGED, pad=3, seed=100 + variant)
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    got = run_gpu(handle, b, force_variant=variant)
    exp = oracle_batch(Ah, Bh, C0, b)
    # canaries (guards between entries and ld padding) are untouched, bitwise
    written = np.zeros(len(C0), dtype=bool)
    for e in range(len(b)):
        entry_view(written, int(b.offC[e]), int(b.m[e]), int(b.n[e]), int(b.ldc[e]))[...] = True
    assert np.array_equal(got[~written].view(np.uint64), C0[~written].view(np.uint64))
    check_entries(got, exp, Ah, Bh, C0, b)


@pytest.mark.parametrize("variant", range(10))
def test_integer_inputs_bitwise(handle, variant):
    b = ragged_batch(RAGGED, pad=1, seed=200 + variant, dist="int")
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    got = run_gpu(handle, b, force_variant=variant)
    exp = oracle_batch(Ah, Bh, C0, b)
    assert np.array_equal(got.view(np.uint64), exp.view(np.uint64))


def test_identity_and_permutation_bitwise(handle):
    rng = np.random.default_rng(3)
    for b_, r in [(64, 16), (100, 8), (257, 33)]:
        for kind in ("eye", "perm"):
            P = np.eye(b_) if kind == "eye" else np.eye(b_)[rng.permutation(b_)]
            Bm = rng.standard_normal((b_, r))
            Cm = rng.standard_normal((b_, r))
            A = torch.tensor(P.ravel(order="F"), device="cuda")
            B = torch.tensor(Bm.ravel(order="F"), device="cuda")
            C = torch.tensor(Cm.ravel(order="F"), device="cuda")
            d = np.zeros(1, dtype=L.DESC_DTYPE)
            d[0] = (A.data_ptr(), B.data_ptr(), C.data_ptr(), b_, r, b_, b_, b_, b_)
            with handle.plan(d) as p:
                p.launch()
                torch.cuda.synchronize()
            got = C.cpu().numpy().reshape(r, b_).T
            assert np.array_equal(got, Cm + P @ Bm)


def test_small_o_form_full_parity(handle):
    """O-form, 64 x C(256x256) += A(256x16) B(16x256), U[-1,1], seed 0."""
    b = W.small_o_form()
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    exp = oracle_batch(Ah, Bh, C0, b)
    dev = b.to("cuda")
    with handle.plan(L.descs_for(dev), use_graph=True) as p:
        p.launch()
        torch.cuda.synchronize()
    got = host(dev.C)
    check_entries(got, exp, Ah, Bh, C0, b)
    dev2 = b.to("cuda")
    with handle.plan(L.descs_for(dev2)) as p:
        p.launch_plain()
        torch.cuda.synchronize()
    assert np.array_equal(host(dev2.C).view(np.uint64), got.view(np.uint64))


def test_small_plan_tiling_choice_keeps_results(handle):
    """A tuned plan of two to eight waves times its tiling against narrower
    64 x 8 tiles and keeps the faster; the non-split tiles give every element
    the same k order, so whichever it keeps, C is bitwise that of the plans
    forced to 64 x 8, 64 x 16 and 64 x 32 tiles, and matches the oracle."""
    b = W.small_o_form()
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    outs = {}
    for name, force in (("tuned", -1), ("64x8", 0), ("64x16", 1), ("64x32", 2)):
        dev = b.to("cuda")
        with handle.plan(L.descs_for(dev), use_graph=True, force_variant=force) as p:
            p.launch()
            torch.cuda.synchronize()
        outs[name] = host(dev.C)
    for name in ("64x8", "64x16", "64x32"):
        assert np.array_equal(outs[name].view(np.uint64), outs["tuned"].view(np.uint64)), name
    check_entries(outs["tuned"], oracle_batch(Ah, Bh, C0, b), Ah, Bh, C0, b)


def test_persistent_plain_graph_bitwise_and_repeatable(handle):
    forms, bs, rs = W.variable_shapes(300, seed=31, bmin=16, bmax=600)
    base = W.variable_batch(forms, bs, rs, seed=31)
    Ah, Bh, C0 = host(base.A), host(base.B), host(base.C)
    outs = {}
    for mode in ("persistent", "graph", "plain", "persistent2"):
        dev = base.to("cuda")
        with handle.plan(L.descs_for(dev), use_graph=(mode == "graph")) as p:
            if mode == "plain":
                p.launch_plain()
            else:
                p.launch()
            torch.cuda.synchronize()
        outs[mode] = host(dev.C)
    for mode in ("graph", "plain", "persistent2"):
        assert np.array_equal(outs[mode].view(np.uint64), outs["persistent"].view(np.uint64)), mode
    exp = oracle_batch(Ah, Bh, C0, base)
    check_entries(outs["persistent"], exp, Ah, Bh, C0, base)


def test_relaunch_accumulates(handle):
    b = ragged_batch([(70, 20, 40)], pad=0, seed=9, dist="int")
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    dev = b.to("cuda")
    with handle.plan(L.descs_for(dev), use_graph=True) as p:
        p.launch()
        p.launch()
        torch.cuda.synchronize()
    once = oracle_batch(Ah, Bh, C0, b)
    twice = oracle_batch(Ah, Bh, once, b)
    assert np.array_equal(host(dev.C).view(np.uint64), twice.view(np.uint64))


def test_uniform_sweep_full_size_sampled(handle):
    """All 18 uniform groups (b in {256,512,1024} x r in {16,32,64} x T/O,
    batch 4096/1024/256) in ONE persistent graph launch, as the benchmark
    times them; sampled outputs against the oracle."""
    batches = [W.uniform_batch(f, b_, r, n, dist="normal", seed=s, device="cuda")
               for f, b_, r, n, s in W.uniform_sweep_groups()]
    descs = np.concatenate([L.descs_for(b) for b in batches])
    samples = [draw_samples(b, 150, seed=i, extra_entries=[0, len(b) - 1]) for i, b in enumerate(batches)]
    c0s = [c0_at(b, s) for b, s in zip(batches, samples)]
    with handle.plan(descs, use_graph=True) as p:
        p.launch()
        torch.cuda.synchronize()
    for b, s, c0 in zip(batches, samples, c0s):
        sample_check(b, b.C, c0, s)


def test_variable_size_full_size_sampled(handle):
    """20,000 entries, b log-uniform in [64, 2048], r in {8,...,128}, T/O
    50/50, operands from a shared 4 GB pool, one graph-captured persistent
    launch with autotuned tiles; sampled outputs (incl. the 50 largest and
    smallest entries) against the oracle."""
    forms, bs, rs = W.variable_shapes(20000, seed=3)
    b = W.variable_batch(forms, bs, rs, seed=3, device="cuda", pool_elems=(4 << 30) // 8)
    flops = 2.0 * b.m * b.n * b.k
    order = np.argsort(flops)
    extra = np.concatenate([order[:50], order[-50:]])
    s = draw_samples(b, 3000, seed=5, extra_entries=extra)
    c0 = c0_at(b, s)
    with handle.plan(L.descs_for(b), use_graph=True) as p:
        p.launch()
        torch.cuda.synchronize()
    sample_check(b, b.C, c0, s)
    del b
    torch.cuda.empty_cache()


def test_execute_host_pipelined_pieces(handle):
    """lrb_execute_host on host buffers: ~200 MB of pinned entries (several
    pipelined pieces, run twice so the cached plans are reused) and pageable
    entries with padded leading dimensions (2-D copies) where two entries
    share one A (copied once); every C against the oracle, padding untouched."""
    big = W.uniform_batch(W.FORM_O, 512, 16, 96, dist="normal", seed=61)          # 96 x 2 MB of C
    Ah, Bh, C0 = host(big.A), host(big.B), host(big.C)
    pinned = [torch.from_numpy(x.copy()).pin_memory() for x in (Ah, Bh, C0)]
    small = ragged_batch([(100, 30, 40), (37, 5, 19), (100, 30, 40)], pad=3, seed=62)
    sA, sB, sC0 = host(small.A), host(small.B), host(small.C)
    sC = sC0.copy()

    def rows(ptrs, b):
        d = np.zeros(len(b), dtype=L.DESC_DTYPE)
        for key, base, off in (("A", ptrs[0], b.offA), ("B", ptrs[1], b.offB), ("C", ptrs[2], b.offC)):
            d[key] = np.uint64(base) + 8 * off.astype(np.uint64)
        for key in ("m", "n", "k", "lda", "ldb", "ldc"):
            d[key] = getattr(b, key)
        return d

    d_big = rows([t.data_ptr() for t in pinned], big)
    d_small = rows([sA.ctypes.data, sB.ctypes.data, sC.ctypes.data], small)
    d_small["A"][2] = d_small["A"][0]              # entry 2 shares entry 0's A
    small_shared = W.Batch(small.A, small.B, small.C, small.m, small.n, small.k, small.lda, small.ldb, small.ldc,
                           np.array([small.offA[0], small.offA[1], small.offA[0]]), small.offB, small.offC)

    handle.execute_host(np.concatenate([d_big, d_small]))
    exp1 = oracle_batch(Ah, Bh, C0, big)
    check_entries(pinned[2].numpy().copy(), exp1, Ah, Bh, C0, big)
    exp_s = oracle_batch(sA, sB, sC0, small_shared)
    check_entries(sC.copy(), exp_s, sA, sB, sC0, small_shared)
    written = np.zeros(len(sC), dtype=bool)
    for e in range(len(small)):
        entry_view(written, int(small.offC[e]), int(small.m[e]), int(small.n[e]), int(small.ldc[e]))[...] = True
    assert np.array_equal(sC[~written].view(np.uint64), sC0[~written].view(np.uint64))

    handle.execute_host(d_big)                     # second call on the big part alone
    handle.execute_host(d_big)                     # and again: cached plans
    exp3 = oracle_batch(Ah, Bh, oracle_batch(Ah, Bh, exp1, big), big)
    check_entries(pinned[2].numpy().copy(), exp3, Ah, Bh, exp1, big, tol=3e-13)


def test_execute_host_timing_summary(handle):
    """lrb_execute_host_get_timing after a timed call: the byte counts are the
    copies the call makes (A, B, C in; C out), every engine's busy time fits
    in the call's span, overlaps are no longer than either engine's busy time,
    and the result is still the oracle's."""
    with L.Handle(0) as h:
        with pytest.raises(L.LrbError):
            h.host_timing()                      # nothing timed yet
        b = W.uniform_batch(W.FORM_T, 512, 32, 256, dist="normal", seed=63)      # ~300 MB, several pieces
        Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
        pinned = [torch.from_numpy(x.copy()).pin_memory() for x in (Ah, Bh, C0)]
        d = np.zeros(len(b), dtype=L.DESC_DTYPE)
        for key, t, off in (("A", pinned[0], b.offA), ("B", pinned[1], b.offB), ("C", pinned[2], b.offC)):
            d[key] = np.uint64(t.data_ptr()) + 8 * off.astype(np.uint64)
        for key in ("m", "n", "k", "lda", "ldb", "ldc"):
            d[key] = getattr(b, key)
        h.set_host_timing(True)
        h.execute_host(d)
        t = h.host_timing()
        assert t["valid"] == 1 and t["pieces"] >= 2
        assert t["h2d_bytes"] == 8 * (Ah.size + Bh.size + C0.size)
        assert t["d2h_bytes"] == 8 * C0.size
        for key in ("h2d_busy_ms", "compute_busy_ms", "d2h_busy_ms"):
            assert 0 < t[key] <= t["wall_ms"] + 1e-6
        assert t["overlap_h2d_compute_ms"] <= min(t["h2d_busy_ms"], t["compute_busy_ms"]) + 1e-6
        assert t["overlap_d2h_compute_ms"] <= min(t["d2h_busy_ms"], t["compute_busy_ms"]) + 1e-6
        assert 0 <= t["compute_start_ms"] <= t["wall_ms"]
        check_entries(pinned[2].numpy().copy(), oracle_batch(Ah, Bh, C0, b), Ah, Bh, C0, b)


def test_execute_host_shared_pool():
    """Entries whose A and B are overlapping views into one pinned host pool
    (the variable-size batch's layout) and whose C are distinct: the pool's
    span is copied once (the byte count says so), the entries keep their
    leading dimensions, and every C matches the oracle; a second call reuses
    the cached layout."""
    forms, bs, rs = W.variable_shapes(120, seed=93, bmin=16, bmax=300)
    b = W.variable_batch(forms, bs, rs, seed=93, pool_elems=1 << 20)
    Ah, C0 = host(b.A), host(b.C)
    pool = torch.from_numpy(Ah.copy()).pin_memory()
    C = torch.from_numpy(C0.copy()).pin_memory()
    d = np.zeros(len(b), dtype=L.DESC_DTYPE)
    d["A"] = np.uint64(pool.data_ptr()) + 8 * b.offA.astype(np.uint64)
    d["B"] = np.uint64(pool.data_ptr()) + 8 * b.offB.astype(np.uint64)
    d["C"] = np.uint64(C.data_ptr()) + 8 * b.offC.astype(np.uint64)
    for key in ("m", "n", "k", "lda", "ldb", "ldc"):
        d[key] = getattr(b, key)
    lo = min(int(b.offA.min()), int(b.offB.min()))
    hi = max(int((b.offA + b.lda.astype(np.int64) * b.k).max()), int((b.offB + b.ldb.astype(np.int64) * b.n).max()))
    with L.Handle(0) as h:
        h.set_host_timing(True)
        h.execute_host(d)
        t = h.host_timing()
        c_elems = int(np.sum(b.m.astype(np.int64) * b.n))
        c_span = int((b.offC + b.ldc.astype(np.int64) * b.n).max() - b.offC.min())
        # the C blocks (and the < 256-byte alignment gaps between them) each way,
        # the pool's span once rather than once per entry
        assert 8 * c_elems <= t["d2h_bytes"] <= 8 * c_span
        assert t["h2d_bytes"] <= 8 * ((hi - lo) + c_span)
        assert t["pieces"] >= 1
        exp1 = oracle_batch(Ah, Ah, C0, b)
        check_entries(C.numpy().copy(), exp1, Ah, Ah, C0, b)
        h.execute_host(d)
        check_entries(C.numpy().copy(), oracle_batch(Ah, Ah, exp1, b), Ah, Ah, exp1, b, tol=3e-13)


def test_multi_plan_two_handles():
    """lrb_multi_plan_create over two handles (both on device 0 here: every
    call of this suite has one GPU) partitions the batch by LPT over 2 m n k,
    each part planned and launched on its own stream with no synchronisation
    between them; every C matches the oracle and the parts' entry counts are
    the partition's."""
    forms, bs, rs = W.variable_shapes(200, seed=91, bmin=16, bmax=600)
    b = W.variable_batch(forms, bs, rs, seed=91)
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    dev = b.to("cuda")
    part, _ = L.lrb_partition_lpt(2.0 * b.m.astype(float) * b.n * b.k, 2)
    with L.Handle(0) as h1, L.Handle(0) as h2:
        with L.MultiPlan([h1, h2], L.descs_for(dev), use_graph=True) as mp:
            assert [mp.part_info(i)["entries"] for i in range(2)] == [int(np.sum(part == i)) for i in range(2)]
            s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
            mp.launch([s1, s2])
            torch.cuda.synchronize()
    check_entries(host(dev.C), oracle_batch(Ah, Bh, C0, b), Ah, Bh, C0, b)


def test_fp64_peak_probe():
    """The FP64-pipe probe reports a rate near the unit-count figure (SMs x 2
    DFMA lanes x 2 flops x clock) at the GPU's clock range, and rejects bad
    arguments."""
    props = torch.cuda.get_device_properties(0)
    tflops, ms = L.lrb_fp64_peak_probe(0, 1 << 16)
    lo = props.multi_processor_count * 2 * 2 * 0.9e9 / 1e12         # at 900 MHz
    hi = props.multi_processor_count * 2 * 2 * 2.2e9 / 1e12 * 1.05  # at 2.2 GHz, 5 % slack
    assert ms > 0 and lo <= tflops <= hi, (tflops, lo, hi)
    with pytest.raises(L.LrbError):
        L.lrb_fp64_peak_probe(0, 0)


def test_allocation_failure_is_reported(handle):
    """A host-buffer batch whose device arena cannot exist (720 GB) fails with
    LRB_ERR_NOMEM before any copy touches the (fake) host pointers."""
    d = np.zeros(1, dtype=L.DESC_DTYPE)
    d[0] = (0x10000000, 0x20000000, 0x30000000, 300000, 300000, 1, 300000, 1, 300000)
    o = L.make_opts(check_alias=False)
    st = L.lib().lrb_execute_host(handle.ptr, d.ctypes.data, 1, ctypes.byref(o), None)
    assert st == L.LRB_ERR_NOMEM
    assert "arena" in L.last_error()
