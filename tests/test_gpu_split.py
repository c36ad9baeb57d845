"""GPU parity of the split-precision (tcgen05) path against the split oracle.

* Exactness invariant: the FP32 level sums the tensor cores leave in TMEM
  for every k-chunk equal the oracle's int64 digit sums, bitwise (this pins
  the digit split, the operand layout and the FP32 accumulation).
* End to end: the GPU result and the oracle's differ only by the grouping of
  exact terms in the binary64 recombination, so |gpu - oracle| <=
  gamma_n (|C0| + sum |terms|) with n the number of binary64 additions.
  Integer inputs are exact on both sides: bitwise.
* Against the exact product (FP64 oracle): within the a-priori bound; the
  relative Frobenius error per digit count is recorded in the test.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import PRESETS
from paper_2311_07602_gb300 import lrbatch as L
from paper_2311_07602_gb300 import workloads as W
from tests.parity import entry_view, host, oracle_batch
from tests.test_gpu_fp64 import ragged_batch

pytestmark = pytest.mark.gpu

PREC = {"bf16_s3": L.LRB_PREC_SPLIT_BF16_S3, "bf16_s4": L.LRB_PREC_SPLIT_BF16_S4,
        "fp16_s3": L.LRB_PREC_SPLIT_FP16_S3, "fp16_s4": L.LRB_PREC_SPLIT_FP16_S4}
# Relative Frobenius error vs the exact product on 10^U(-4,4) N(0,1) data,
# upper limits, above the errors measured on the GB300.
WIDE_REL_ERR = {"bf16_s3": 3e-6, "bf16_s4": 1e-8, "fp16_s3": 3e-7, "fp16_s4": 1e-9}


@pytest.fixture(scope="module")
def handle():
    h = L.Handle(0)
    yield h
    h.close()


def mats(batch, e, Ah, Bh, Ch):
    m, n, k = int(batch.m[e]), int(batch.n[e]), int(batch.k[e])
    A = entry_view(Ah, int(batch.offA[e]), m, k, int(batch.lda[e])).copy()
    B = entry_view(Bh, int(batch.offB[e]), k, n, int(batch.ldb[e])).copy()
    C = entry_view(Ch, int(batch.offC[e]), m, n, int(batch.ldc[e])).copy()
    return A, B, C


def wide(batch):
    rng = np.random.default_rng(int(batch.m.sum()))
    for t in (batch.A, batch.B):
        x = t.numpy()
        fin = np.isfinite(x)
        x[fin] *= 10.0 ** rng.uniform(-4, 4, int(fin.sum()))
    return batch


def plant_special_rows(b, p):
    """Rows of A that exercise every branch of the digit extraction: a zero
    row, rows of values below 2^-997 in one chunk only (the exact 64-bit path;
    one subnormal), exact half-unit ties of the rounding, and a row maximum
    just below a power of two (its top digit rounds up to 2^beta)."""
    A = entry_view(b.A.numpy(), int(b.offA[0]), int(b.m[0]), int(b.k[0]), int(b.lda[0]))
    kc = p.kc
    A[3, :] = 0.0
    A[5, kc:2 * kc] = np.random.default_rng(1).standard_normal(kc) * 1e-305
    A[5, kc + 7] = 5e-324
    E = 3                                   # ties: (Z + 1/2) 2^(E - beta S) with |values| < 2^E
    Z = np.arange(1, 40) * 977
    A[9, :] = 0.0                           # nothing else in the row, so the chunk maximum is the one below
    A[9, :len(Z)] = np.ldexp(Z + 0.5, E - p.beta * p.S)
    A[9, 50] = np.ldexp(1.0, E) * (1 - 2.0 ** -40)
    A[11, :] = np.ldexp(1.0 - 2.0 ** -53, 2) * np.sign(np.random.default_rng(2).standard_normal(A.shape[1]))
    return b


def plant_special_cols(b, p):
    """The same cases in columns of B, which the pre-pass slices column by
    column: a zero column, a column of values below 2^-997 in one chunk only
    (one subnormal), exact half-unit ties, and a column maximum just below a
    power of two."""
    B = entry_view(b.B.numpy(), int(b.offB[0]), int(b.k[0]), int(b.n[0]), int(b.ldb[0]))
    kc = p.kc
    B[:, 3] = 0.0
    B[kc:2 * kc, 5] = np.random.default_rng(3).standard_normal(kc) * 1e-305
    B[kc + 7, 5] = 5e-324
    E = 3
    Z = np.arange(1, 40) * 613
    B[:, 9] = 0.0
    B[:len(Z), 9] = np.ldexp(Z + 0.5, E - p.beta * p.S)
    B[50, 9] = np.ldexp(1.0, E) * (1 - 2.0 ** -40)
    B[:, 11] = np.ldexp(1.0 - 2.0 ** -53, 2) * np.sign(np.random.default_rng(4).standard_normal(B.shape[0]))
    return b


@pytest.mark.parametrize("name", sorted(PREC))
@pytest.mark.parametrize("n", [70, 40])
def test_level_sums_bitwise(handle, name, n):
    # n = 70: several column tiles, both operands sliced by the pre-passes;
    # n = 40: one column tile, A sliced inside the kernel; B always by the
    # pre-pass (the 32-bit digit path for BF16 S = 3 wherever a row or column
    # allows it, with the special rows and columns below)
    p = PRESETS[name]
    b = plant_special_cols(plant_special_rows(wide(ragged_batch([(150, n, 2 * p.kc + 44)], pad=2, seed=7)), p), p)
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    A, B, _ = mats(b, 0, Ah, Bh, C0)
    m, n, k = A.shape[0], B.shape[1], A.shape[1]
    chunks = (k + p.kc - 1) // p.kc
    dev = b.to("cuda")
    dump = torch.zeros(chunks * p.S * m * n, dtype=torch.float32, device="cuda")
    with handle.plan(L.descs_for(dev), precision=PREC[name]) as plan:
        plan.dump_levels(dump.data_ptr())
        assert plan.status() == L.LRB_OK
    got = dump.cpu().numpy().reshape(chunks, p.S, m, n)
    for c in range(chunks):
        _, _, levels = oracle.chunk_level_sums(A, B, p, c)
        for Lv, P in levels.items():
            g = got[c, Lv - 2]
            assert np.all(g == np.rint(g)), "non-integer level sum"
            assert np.array_equal(g.astype(np.int64), P), f"chunk {c} level {Lv}"


SHAPES = [(1, 1, 1), (128, 64, 128), (129, 65, 129), (300, 64, 300), (256, 256, 64), (70, 200, 16), (64, 8, 1000)]


@pytest.mark.parametrize("name", sorted(PREC))
def test_matches_split_oracle(handle, name):
    p = PRESETS[name]
    b = wide(ragged_batch(SHAPES, pad=3, seed=21))
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    dev = b.to("cuda")
    with handle.plan(L.descs_for(dev), precision=PREC[name]) as plan:
        plan.launch()
        assert plan.status() == L.LRB_OK
    got = host(dev.C)
    written = np.zeros(len(C0), dtype=bool)
    for e in range(len(b)):
        A, B, C = mats(b, e, Ah, Bh, C0)
        exp = oracle.split_gemm(A, B, C, p)
        g = entry_view(got, int(b.offC[e]), *C.shape, int(b.ldc[e]))
        entry_view(written, int(b.offC[e]), *C.shape, int(b.ldc[e]))[...] = True
        nadd = ((A.shape[1] + p.kc - 1) // p.kc) * (len(p.levels()) + 1)
        tol = 2 * oracle.gamma(nadd) * oracle.recombination_magnitude(A, B, C, p)
        assert np.all(np.abs(g - exp) <= tol), f"entry {e} {A.shape}x{B.shape}"
        # and against the exact product, within the a-priori bound
        exact_bound = oracle.apriori_bound(A, B, C, p)
        ref = C + A @ B
        assert np.all(np.abs(g - ref) <= exact_bound + 4 * oracle.gamma(A.shape[1] + 2) *
                      (np.abs(C) + np.abs(A) @ np.abs(B)))
    assert np.array_equal(got[~written].view(np.uint64), C0[~written].view(np.uint64))


@pytest.mark.parametrize("name", sorted(PREC))
def test_integer_inputs_exact(handle, name):
    b = ragged_batch(SHAPES, pad=1, seed=5, dist="int")
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    exp = oracle_batch(Ah, Bh, C0, b)
    dev = b.to("cuda")
    with handle.plan(L.descs_for(dev), precision=PREC[name]) as plan:
        plan.launch()
        assert plan.status() == L.LRB_OK
    assert np.array_equal(host(dev.C).view(np.uint64), exp.view(np.uint64))


@pytest.mark.parametrize("name", sorted(PREC))
def test_wide_range_error_vs_exact(handle, name):
    p = PRESETS[name]
    errs = []
    for form in (W.FORM_T, W.FORM_O):
        b = W.wide_range(form, batch=3, b=256, r=64, seed=40 + form)
        Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
        dev = b.to("cuda")
        with handle.plan(L.descs_for(dev), precision=PREC[name]) as plan:
            plan.launch()
            assert plan.status() == L.LRB_OK
        got = host(dev.C)
        ref = oracle_batch(Ah, Bh, np.zeros_like(C0), b)   # A B alone, binary64
        for e in range(len(b)):
            A, B, C = mats(b, e, Ah, Bh, C0)
            g = entry_view(got, int(b.offC[e]), *C.shape, int(b.ldc[e])) - C
            r = entry_view(ref, int(b.offC[e]), *C.shape, int(b.ldc[e]))
            errs.append(np.linalg.norm(g - r) / np.linalg.norm(r))
    assert max(errs) <= WIDE_REL_ERR[name], f"{name}: {max(errs):.3e}"


@pytest.mark.parametrize("name", ["bf16_s3", "bf16_s4"])
@pytest.mark.parametrize("form", [W.FORM_T, W.FORM_O])
def test_full_size_sampled(handle, name, form):
    """b = 1024, r = 64, batch 2048, entries 10^U(-4,4) N(0,1): one launch,
    sampled outputs against the split oracle's element sampler."""
    p = PRESETS[name]
    b = W.wide_range(form, batch=2048, device="cuda")
    rng = np.random.default_rng(3)
    q = 400
    ents = np.concatenate([rng.integers(0, len(b), q), [0, len(b) - 1]])
    ii = (rng.random(len(ents)) * b.m[ents]).astype(np.int64)
    jj = (rng.random(len(ents)) * b.n[ents]).astype(np.int64)
    k = int(b.k[0])
    pk = np.arange(k)
    a_idx = b.offA[ents][:, None] + ii[:, None] + pk[None, :] * b.lda[ents][:, None]
    b_idx = b.offB[ents][:, None] + pk[None, :] + jj[:, None] * b.ldb[ents][:, None]
    c_idx = b.offC[ents] + ii + jj * b.ldc[ents]
    arow = b.A[torch.as_tensor(a_idx.ravel(), device="cuda")].cpu().numpy().reshape(len(ents), k)
    bcol = b.B[torch.as_tensor(b_idx.ravel(), device="cuda")].cpu().numpy().reshape(len(ents), k)
    c0 = b.C[torch.as_tensor(c_idx, device="cuda")].cpu().numpy()
    with handle.plan(L.descs_for(b), precision=PREC[name]) as plan:
        plan.launch()
        assert plan.status() == L.LRB_OK
    got = b.C[torch.as_tensor(c_idx, device="cuda")].cpu().numpy()
    exp = oracle.split_dot_samples(arow, bcol, c0, p)
    mag = np.abs(c0) + np.sum(np.abs(arow) * np.abs(bcol), axis=1)
    nadd = ((k + p.kc - 1) // p.kc) * (len(p.levels()) + 1)
    assert np.all(np.abs(got - exp) <= 4 * oracle.gamma(nadd) * mag)
    del b
    torch.cuda.empty_cache()


@pytest.mark.parametrize("shapes", [[(128, 64, 130), (100, 64, 200)], [(200, 130, 64), (100, 90, 70)]],
                         ids=["one-column-tile", "pre-sliced-A"])
def test_bounded_wait_expiry_reports_timeout(handle, shapes):
    """Failure path without a GPU fault: with test_stall the kernel also waits
    on a barrier nothing arrives on; its 2 s bound expires, it drains its own
    tensor-core work and its copies in flight, frees TMEM, leaves its C tiles
    unwritten and sets the plan's status word; the context stays usable for
    the next plan.  The second batch's entries have several column tiles, so
    A comes pre-sliced and its units arrive by bulk copies."""
    b = wide(ragged_batch(shapes, pad=0, seed=71))
    Ah, Bh, C0 = host(b.A), host(b.B), host(b.C)
    dev = b.to("cuda")
    with handle.plan(L.descs_for(dev), precision=PREC["bf16_s3"], test_stall=True) as plan:
        plan.launch()
        assert plan.status() == L.LRB_ERR_TIMEOUT
    assert np.array_equal(host(dev.C).view(np.uint64), C0.view(np.uint64))
    dev2 = b.to("cuda")
    with handle.plan(L.descs_for(dev2), precision=PREC["bf16_s3"]) as plan:
        plan.launch()
        assert plan.status() == L.LRB_OK
    p = PRESETS["bf16_s3"]
    got = host(dev2.C)
    for e in range(len(b)):
        A, B, C = mats(b, e, Ah, Bh, C0)
        exp = oracle.split_gemm(A, B, C, p)
        g = entry_view(got, int(b.offC[e]), *C.shape, int(b.ldc[e]))
        nadd = ((A.shape[1] + p.kc - 1) // p.kc) * (len(p.levels()) + 1)
        assert np.all(np.abs(g - exp) <= 2 * oracle.gamma(nadd) * oracle.recombination_magnitude(A, B, C, p))
