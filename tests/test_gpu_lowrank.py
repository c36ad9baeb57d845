"""GPU parity of the low-rank producers and consumers against the oracle
(oracle/lowrank.py and the FP64 GEMM oracle), through the C ABI.

* transposed / overwriting GEMM forms: every (trans, overwrite) pair on
  ragged shapes with ld padding; rel. Frobenius <= 1e-13 and Higham's bound
  per element, bitwise on integer data, C never read when overwriting (its
  window starts as NaN), padding untouched;
* randomized SVD: inputs with a known spectrum and a gap at the kept rank
  r, so the rank-r result is well conditioned: S within 1e-12 sigma_0 of the
  oracle's (and of the chosen spectrum where the block has rank <= l),
  U diag(S) V within 1e-11 ||A||_F of the oracle's, U and V orthonormal to
  1e-13; exact recovery of rank <= l blocks; the zero block; mixed shapes and
  0..3 power iterations in one plan; kernel-matrix blocks at the benchmark's
  size on sampled entries, where the GPU's error must match the oracle's;
* expansion: bitwise on integer data, Higham's bound on random data;
* rounded addition: exact singular values of sums built from disjoint parts
  of one orthonormal pair, reconstruction within 1e-11 of the oracle's, and
  two parts 1e-28 apart (rotations outside binary32's range).
Tolerances: the oracle and the GPU take the same steps with different
summation orders and a different (but backward-stable) QR and SVD; with a
gap g = sigma_r / sigma_{r+1} >= 100 the rank-r truncation moves by about
u ||A|| sqrt(m n) / (1 - 1/g) ~ 1e-13 ||A||, so 1e-11 leaves a margin of 100."""
import numpy as np
import pytest
import torch

import oracle
from oracle import lowrank as OL
from paper_2311_07602_gb300 import lrbatch as L
from paper_2311_07602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    h = L.Handle(0)
    yield h
    h.close()


class DevMat:
    """A column-major matrix on the device with ld = rows + pad; the padding
    (and, for outputs, the window) starts as NaN canaries."""

    def __init__(self, rows, cols, pad=2, value=None):
        self.rows, self.cols, self.ld = rows, cols, rows + pad
        host = np.full(self.ld * cols, np.nan)
        if value is not None:
            self.view(host)[...] = value
        self.host0 = host.copy()
        self.t = torch.from_numpy(host).to("cuda")

    def view(self, flat):
        it = flat.itemsize
        return np.lib.stride_tricks.as_strided(flat, shape=(self.rows, self.cols), strides=(it, it * self.ld))

    @property
    def ptr(self):
        return self.t.data_ptr()

    def get(self):
        flat = self.t.cpu().numpy()
        mask = np.ones(len(flat), dtype=bool)
        self.view(mask)[...] = False
        assert np.array_equal(flat[mask], self.host0[mask], equal_nan=True), "padding was written"
        return np.array(self.view(flat))


def orthonormal(rng, rows, cols):
    Q, _ = np.linalg.qr(rng.standard_normal((rows, cols)))
    return Q


def gapped(rng, m, n, r, tail_rank=None):
    """A = P diag(sigma) Q^T with sigma_0..r-1 in [1, 0.01] and a tail 100x
    below sigma_{r-1}; returns (A, sigma)."""
    k = min(m, n) if tail_rank is None else min(tail_rank, min(m, n))
    head = np.logspace(0, -2, r)
    tail = 1e-4 * np.logspace(0, -3, k - r) if k > r else np.zeros(0)
    sigma = np.concatenate([head, tail])
    A = (orthonormal(rng, m, k) * sigma) @ orthonormal(rng, n, k).T
    return A, sigma


# ------------------------------------------------------ transposed GEMM forms

SHAPES = [(70, 33, 45), (129, 8, 300), (5, 100, 17), (64, 64, 64), (1, 1, 1), (200, 40, 3)]


@pytest.mark.parametrize("overwrite", [False, True])
@pytest.mark.parametrize("trans", [0, 1, 2, 3])
def test_gemm_forms_match_oracle(handle, trans, overwrite):
    rng = np.random.default_rng(10 * trans + overwrite)
    descs, cases = [], []
    for (m, n, k) in SHAPES:
        integer = len(cases) % 2 == 1
        draw = (lambda s: rng.integers(-8, 9, s).astype(float)) if integer else rng.standard_normal
        Aop, Bop = draw((m, k)), draw((k, n))
        C0 = None if overwrite else draw((m, n))
        A = DevMat(*(Aop.T.shape if trans & 1 else Aop.shape), value=Aop.T if trans & 1 else Aop)
        B = DevMat(*(Bop.T.shape if trans & 2 else Bop.shape), value=Bop.T if trans & 2 else Bop)
        C = DevMat(m, n, value=C0)           # overwrite: the window stays NaN, so reading it would show
        descs.append((A.ptr, B.ptr, C.ptr, m, n, k, A.ld, B.ld, C.ld))
        cases.append((Aop, Bop, C0, C, integer, A, B))      # A, B kept alive until the launch is done
    d = np.array(descs, dtype=L.DESC_DTYPE)
    with L.Plan(handle, d, trans=trans, overwrite=overwrite) as p:
        p.launch()
        torch.cuda.synchronize()
        if trans or overwrite:          # only the plain A B (+C) form has the per-shape comparator launch
            with pytest.raises(L.LrbError):
                p.launch_plain()
    for Aop, Bop, C0, C, integer, _, _ in cases:
        m, n, k = Aop.shape[0], Bop.shape[1], Aop.shape[1]
        base = np.zeros((m, n)) if C0 is None else C0
        exp = np.ascontiguousarray(base.ravel(order="F"))
        oracle.gemm(m, n, k, np.ascontiguousarray(Aop.ravel(order="F")), 0, m,
                    np.ascontiguousarray(Bop.ravel(order="F")), 0, k, exp, 0, m)
        exp = exp.reshape(n, m).T
        got = C.get()
        if integer:
            assert np.array_equal(got, exp)
        else:
            assert np.linalg.norm(got - exp) <= 1e-13 * np.linalg.norm(exp)
            lim = 2 * oracle.gamma(k + 1) * (np.abs(base) + np.abs(Aop) @ np.abs(Bop)) * (1 + 2.0 ** -50)
            assert np.all(np.abs(got - exp) <= lim)


def test_gemm_forms_rejected_where_unsupported(handle):
    A, B, C = DevMat(8, 8, value=np.eye(8)), DevMat(8, 8, value=np.eye(8)), DevMat(8, 8, value=np.zeros((8, 8)))
    d = np.array([(A.ptr, B.ptr, C.ptr, 8, 8, 8, A.ld, B.ld, C.ld)], dtype=L.DESC_DTYPE)
    with pytest.raises(L.LrbError) as e:
        L.Plan(handle, d, trans=1, precision=L.LRB_PREC_SPLIT_BF16_S3)
    assert e.value.status == L.LRB_ERR_UNSUPPORTED


# ------------------------------------------------------------ randomized SVD

def rsvd_gpu(handle, blocks, q):
    """blocks: list of (A, Omega, r).  Returns [(U, S, V)] and the plan status."""
    keep, descs = [], []
    for A, Om, r in blocks:
        m, n = A.shape
        l = Om.shape[1]
        dA, dO = DevMat(m, n, value=A), DevMat(n, l, value=Om)
        dU, dS, dV = DevMat(m, r), DevMat(r, 1, pad=0), DevMat(r, n)
        keep.append((dA, dO, dU, dS, dV))
        descs.append((dA.ptr, dO.ptr, (dU.ptr, dS.ptr, dV.ptr, m, n, r, dU.ld, dV.ld, 0), l, dA.ld, dO.ld, 0))
    d = np.array(descs, dtype=L.RSVD_DESC_DTYPE)
    with L.LowRankPlan(handle, "rsvd", d, power_iters=q) as p:
        p.launch()
        st = p.status()
    outs = [(dU.get(), dS.get()[:, 0], dV.get()) for _, _, dU, dS, dV in keep]
    for (A, _, _), (dA, *_ ) in zip(blocks, keep):
        assert np.array_equal(dA.get(), A)           # input untouched
    return outs, st


def check_factors(U, S, V, tol=1e-13):
    r = len(S)
    assert np.all(S[:-1] >= S[1:]) and np.all(S >= 0)
    assert np.abs(U.T @ U - np.eye(r)).max() <= tol
    assert np.abs(V @ V.T - np.eye(r)).max() <= tol


# (m, n, l, r); odd l (13, 27, 33, 1) exercises the SVD core's bye column and odd leading dimension
CASES = [(200, 150, 20, 12), (64, 300, 26, 16), (333, 257, 40, 32), (97, 61, 8, 1), (96, 96, 96, 40),
         (1024, 160, 42, 32), (50, 2000, 18, 8), (150, 120, 13, 5), (300, 200, 27, 16), (65, 70, 33, 20),
         (40, 45, 1, 1)]


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rsvd_gapped_spectrum(handle, q):
    rng = np.random.default_rng(100 + q)
    blocks, sig = [], []
    for (m, n, l, r) in CASES:
        A, sigma = gapped(rng, m, n, r)
        blocks.append((A, rng.standard_normal((n, l)), r))
        sig.append(sigma)
    outs, st = rsvd_gpu(handle, blocks, q)
    assert st == L.LRB_OK
    for (A, Om, r), (U, S, V), sigma in zip(blocks, outs, sig):
        Uo, So, Vo = OL.rsvd(A, Om, r, q)
        assert np.abs(S - So).max() <= 1e-12 * sigma[0]
        X, Xo = (U * S) @ V, (Uo * So) @ Vo
        assert np.linalg.norm(X - Xo) <= 1e-11 * np.linalg.norm(A), (A.shape, r)
        check_factors(U, S, V)


def test_rsvd_exact_rank_and_known_values(handle):
    rng = np.random.default_rng(7)
    blocks, want = [], []
    for (m, n, k, l, r) in [(150, 120, 6, 10, 6), (300, 64, 16, 26, 16), (77, 77, 9, 9, 5)]:
        sigma = 2.0 ** -np.arange(k)
        A = (orthonormal(rng, m, k) * sigma) @ orthonormal(rng, n, k).T
        blocks.append((A, rng.standard_normal((n, l)), r))
        want.append(sigma)
    outs, st = rsvd_gpu(handle, blocks, 0)
    assert st == L.LRB_OK
    for (A, Om, r), (U, S, V), sigma in zip(blocks, outs, want):
        assert np.abs(S - sigma[:r]).max() <= 1e-13 * sigma[0]
        if r == len(sigma):
            assert np.linalg.norm((U * S) @ V - A) <= 1e-13 * np.linalg.norm(A)
        check_factors(U, S, V)


def test_rsvd_zero_block(handle):
    rng = np.random.default_rng(3)
    A = np.zeros((90, 70))
    (U, S, V), = rsvd_gpu(handle, [(A, rng.standard_normal((70, 12)), 5)], 1)[0]
    assert np.all(S == 0.0)
    assert np.all((U * S) @ V == 0.0)
    # a zero singular value gives a zero row of V; U keeps orthonormal columns
    assert np.all(V == 0.0)
    assert np.abs(U.T @ U - np.eye(5)).max() <= 1e-15


def test_rsvd_mixed_shapes_one_plan(handle):
    rng = np.random.default_rng(11)
    blocks = []
    for (m, n, l, r) in [(512, 512, 26, 16), (64, 64, 64, 64), (100, 300, 12, 3), (700, 90, 40, 30), (33, 33, 5, 5)]:
        A, _ = gapped(rng, m, n, r)
        blocks.append((A, rng.standard_normal((n, l)), r))
    for q in (0, 3):
        outs, st = rsvd_gpu(handle, blocks, q)
        assert st == L.LRB_OK
        for (A, Om, r), (U, S, V) in zip(blocks, outs):
            Uo, So, Vo = OL.rsvd(A, Om, r, q)
            assert np.linalg.norm((U * S) @ V - (Uo * So) @ Vo) <= 1e-11 * np.linalg.norm(A)


def test_rsvd_validation(handle):
    dA, dO = DevMat(40, 30, value=np.ones((40, 30))), DevMat(30, 10, value=np.ones((30, 10)))
    dU, dS, dV = DevMat(40, 8), DevMat(8, 1, pad=0), DevMat(8, 30)

    def desc(**kw):
        f = dict(A=dA.ptr, O=dO.ptr, U=dU.ptr, S=dS.ptr, V=dV.ptr, m=40, n=30, r=8, ldu=dU.ld, ldv=dV.ld,
                 l=10, lda=dA.ld, ldo=dO.ld)
        f.update(kw)
        return np.array([(f["A"], f["O"], (f["U"], f["S"], f["V"], f["m"], f["n"], f["r"], f["ldu"], f["ldv"], 0),
                          f["l"], f["lda"], f["ldo"], 0)], dtype=L.RSVD_DESC_DTYPE)

    def status(q=0, **kw):
        try:
            L.LowRankPlan(handle, "rsvd", desc(**kw), power_iters=q).close()
            return L.LRB_OK
        except L.LrbError as e:
            return e.status

    assert status() == L.LRB_OK
    assert status(l=31) == L.LRB_ERR_INVALID           # l > min(m, n)
    assert status(r=11) == L.LRB_ERR_INVALID           # r > l
    assert status(lda=39) == L.LRB_ERR_INVALID
    assert status(q=9) == L.LRB_ERR_INVALID
    assert status(U=dA.ptr) == L.LRB_ERR_ALIAS          # output over the input
    assert status(V=dU.ptr) == L.LRB_ERR_ALIAS          # two outputs overlap
    assert status(U=dU.ptr + 4) == L.LRB_ERR_INVALID    # misaligned
    assert status(m=9000, lda=9000, ldu=9000) == L.LRB_ERR_UNSUPPORTED
    big = DevMat(200, 100, value=np.zeros((200, 100)))
    assert status(A=big.ptr, m=200, n=100, lda=big.ld, l=97, r=8, O=big.ptr, ldo=big.ld,
                  U=DevMat(200, 8).ptr, ldu=202) == L.LRB_ERR_UNSUPPORTED   # l above the limit


def test_rsvd_kernel_blocks_benchmark_size(handle):
    """The benchmark's shape (1024 x 1024 kernel-matrix blocks, r = 16, l = 26,
    q = 1) in one plan of 64 blocks; three sampled blocks against the oracle:
    the GPU's approximation error matches the oracle's, and so do the factors."""
    count, b, r, l, q = 64, 1024, 16, 26, 1
    A = W.kernel_blocks(count, b, b, seed=7, device="cuda")
    Om = W.gaussian_test_matrix(b, l, seed=8, device="cuda")
    U = torch.full((count * b * r,), float("nan"), dtype=torch.float64, device="cuda")
    S = torch.full((count * r,), float("nan"), dtype=torch.float64, device="cuda")
    V = torch.full((count * r * b,), float("nan"), dtype=torch.float64, device="cuda")
    d = np.zeros(count, dtype=L.RSVD_DESC_DTYPE)
    e = np.arange(count, dtype=np.uint64)
    d["A"] = np.uint64(A.data_ptr()) + np.uint64(8 * b * b) * e
    d["Omega"] = Om.data_ptr()
    d["out"]["U"] = np.uint64(U.data_ptr()) + np.uint64(8 * b * r) * e
    d["out"]["S"] = np.uint64(S.data_ptr()) + np.uint64(8 * r) * e
    d["out"]["V"] = np.uint64(V.data_ptr()) + np.uint64(8 * r * b) * e
    d["out"]["m"], d["out"]["n"], d["out"]["r"], d["out"]["ldu"], d["out"]["ldv"] = b, b, r, b, r
    d["l"], d["lda"], d["ldo"] = l, b, b
    with L.LowRankPlan(handle, "rsvd", d, power_iters=q) as p:
        p.launch()
        assert p.status() == L.LRB_OK
    Ah, Oh = A.cpu().numpy(), Om.cpu().numpy().reshape(l, b).T
    Uh, Sh, Vh = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    for e in (0, 31, 63):
        Ae = Ah[e * b * b:(e + 1) * b * b].reshape(b, b).T
        Ue = Uh[e * b * r:(e + 1) * b * r].reshape(r, b).T
        Se = Sh[e * r:(e + 1) * r]
        Ve = Vh[e * r * b:(e + 1) * r * b].reshape(b, r).T
        Uo, So, Vo = OL.rsvd(Ae, Oh, r, q)
        err_gpu = np.linalg.norm(Ae - (Ue * Se) @ Ve)
        err_ora = np.linalg.norm(Ae - (Uo * So) @ Vo)
        nA = np.linalg.norm(Ae)
        assert err_gpu <= err_ora * (1 + 1e-6) + 1e-12 * nA
        assert np.abs(Se - So).max() <= 1e-12 * So[0]
        assert np.linalg.norm((Ue * Se) @ Ve - (Uo * So) @ Vo) <= 1e-10 * nA
        check_factors(Ue, Se, Ve, tol=1e-12)


# --------------------------------------------------------------- expansion

def test_expand_matches_oracle(handle):
    rng = np.random.default_rng(5)
    keep, descs = [], []
    for i, (m, n, r) in enumerate([(100, 80, 8), (257, 129, 16), (33, 500, 1), (64, 64, 64)]):
        integer = i % 2 == 0
        draw = (lambda s: rng.integers(-6, 7, s).astype(float)) if integer else rng.standard_normal
        U, S, V, D0 = draw((m, r)), draw(r), draw((r, n)), draw((m, n))
        dU, dS, dV, dD = DevMat(m, r, value=U), DevMat(r, 1, pad=0, value=S[:, None]), DevMat(r, n, value=V), \
            DevMat(m, n, value=D0)
        keep.append((U, S, V, D0, dD, integer))
        descs.append(((dU.ptr, dS.ptr, dV.ptr, m, n, r, dU.ld, dV.ld, 0), dD.ptr, dD.ld, 0))
        keep[-1] = keep[-1] + ((dU, dS, dV),)
    d = np.array(descs, dtype=L.EXPAND_DESC_DTYPE)
    with L.LowRankPlan(handle, "expand", d) as p:
        p.launch()
        assert p.status() == L.LRB_OK
    for U, S, V, D0, dD, integer, _ in keep:
        exp = OL.lr_expand(U, S, V, D0)
        got = dD.get()
        if integer:
            assert np.array_equal(got, exp)
        else:
            r = len(S)
            lim = 2 * oracle.gamma(r + 2) * (np.abs(D0) + np.abs(U * S) @ np.abs(V)) * (1 + 2.0 ** -50)
            assert np.all(np.abs(got - exp) <= lim)


# -------------------------------------------------------- rounded addition

def round_add_gpu(handle, items):
    """items: list of ((U1, S1, V1), (U2, S2, V2), r) -> [(U, S, V)]."""
    keep, descs = [], []
    for (x, y, r) in items:
        m, n = x[0].shape[0], x[2].shape[1]
        blk = []
        for (U, S, V) in (x, y):
            dU, dS, dV = DevMat(m, len(S), value=U), DevMat(len(S), 1, pad=0, value=S[:, None]), \
                DevMat(len(S), n, value=V)
            blk.append((dU, dS, dV))
        oU, oS, oV = DevMat(m, r), DevMat(r, 1, pad=0), DevMat(r, n)
        keep.append((blk, (oU, oS, oV)))
        row = []
        for (dU, dS, dV) in blk + [(oU, oS, oV)]:
            row.append((dU.ptr, dS.ptr, dV.ptr, m, n, dU.cols, dU.ld, dV.ld, 0))
        descs.append(tuple(row))
    d = np.array(descs, dtype=L.ROUND_ADD_DESC_DTYPE)
    with L.LowRankPlan(handle, "round_add", d) as p:
        p.launch()
        assert p.status() == L.LRB_OK
    return [(oU.get(), oS.get()[:, 0], oV.get()) for _, (oU, oS, oV) in keep]


def test_round_add_known_spectrum(handle):
    rng = np.random.default_rng(31)
    items, want = [], []
    for (m, n, r1, r2, r) in [(200, 150, 8, 8, 8), (96, 300, 16, 20, 24), (64, 64, 32, 32, 64), (50, 40, 3, 1, 2),
                              (150, 130, 5, 8, 7), (90, 80, 1, 2, 2)]:
        P, Q = orthonormal(rng, m, r1 + r2), orthonormal(rng, n, r1 + r2)
        s = rng.permutation(np.logspace(0, -3, r1 + r2))
        x = (P[:, :r1], s[:r1], Q[:, :r1].T.copy())
        y = (P[:, r1:], s[r1:], Q[:, r1:].T.copy())
        items.append((x, y, r))
        want.append(np.sort(s)[::-1])
    outs = round_add_gpu(handle, items)
    for (x, y, r), (U, S, V), allv in zip(items, outs, want):
        assert np.abs(S - allv[:r]).max() <= 1e-13 * allv[0]
        Uo, So, Vo = OL.lr_round_add(*x, *y, r)
        assert np.linalg.norm((U * S) @ V - (Uo * So) @ Vo) <= 1e-12 * allv[0] * np.sqrt(r)
        check_factors(U, S, V)


def test_round_add_extremely_graded_spectrum(handle):
    """Two blocks 28 orders of magnitude apart.  The SVD core's QR leaves
    columns whose norms differ by ~1e-28, where zeta = (b - a) / 2g of a
    rotation is far outside binary32's range; such pairs must still be
    rotated (in binary64), or V keeps rows at an O(1) angle."""
    rng = np.random.default_rng(33)
    m, n, r1, r2 = 120, 90, 10, 6
    P, Q = orthonormal(rng, m, r1 + r2), orthonormal(rng, n, r1 + r2)
    x = (P[:, :r1], np.logspace(0, -2, r1), Q[:, :r1].T.copy())
    y = (P[:, r1:], 1e-28 * np.logspace(0, -2, r2), Q[:, r1:].T.copy())
    r = r1 + r2
    (U, S, V), = round_add_gpu(handle, [(x, y, r)])
    check_factors(U, S, V)
    allv = np.sort(np.concatenate([x[1], y[1]]))[::-1]
    assert np.abs(S - allv).max() <= 1e-13
    dense = (x[0] * x[1]) @ x[2] + (y[0] * y[1]) @ y[2]
    assert np.linalg.norm((U * S) @ V - dense) <= 1e-13 * np.linalg.norm(dense)


def test_round_add_benchmark_size_sampled(handle):
    """512 rounded additions of 1024 x 1024 rank-16 blocks in one plan (the
    benchmark's launch); y is 1e-5 below x, so the rank-16 truncation has a
    gap and is well conditioned.  Pairs 0, 255 and 511 against the oracle."""
    rng = np.random.default_rng(35)
    m = n = 1024
    r, cnt = 16, 512
    items = []
    for _ in range(cnt):
        x = (rng.standard_normal((m, r)) / np.sqrt(m), np.logspace(0, -2, r), rng.standard_normal((r, n)) / np.sqrt(n))
        y = (rng.standard_normal((m, r)) / np.sqrt(m), 1e-5 * np.logspace(0, -2, r),
             rng.standard_normal((r, n)) / np.sqrt(n))
        items.append((x, y, r))
    outs = round_add_gpu(handle, items)
    for e in (0, 255, 511):
        (x, y, _), (U, S, V) = items[e], outs[e]
        Uo, So, Vo = OL.lr_round_add(*x, *y, r)
        dense = (x[0] * x[1]) @ x[2] + (y[0] * y[1]) @ y[2]
        assert np.abs(S - So).max() <= 1e-12 * So[0], e
        assert np.linalg.norm((U * S) @ V - (Uo * So) @ Vo) <= 1e-11 * np.linalg.norm(dense), e
        check_factors(U, S, V)


def test_round_add_random_matches_oracle(handle):
    rng = np.random.default_rng(32)
    items = []
    for (m, n, r1, r2, r) in [(300, 200, 16, 16, 16), (128, 1000, 8, 24, 32), (77, 65, 5, 7, 12)]:
        x = (orthonormal(rng, m, r1), np.logspace(0, -2, r1), orthonormal(rng, n, r1).T.copy())
        y = (orthonormal(rng, m, r2), np.logspace(-1, -6, r2), orthonormal(rng, n, r2).T.copy())
        items.append((x, y, r))
    outs = round_add_gpu(handle, items)
    for (x, y, r), (U, S, V) in zip(items, outs):
        Uo, So, Vo = OL.lr_round_add(*x, *y, r)
        dense = (x[0] * x[1]) @ x[2] + (y[0] * y[1]) @ y[2]
        assert np.abs(S - So).max() <= 1e-12 * So[0]
        assert np.linalg.norm((U * S) @ V - (Uo * So) @ Vo) <= 1e-11 * np.linalg.norm(dense)
        if r == len(x[1]) + len(y[1]):
            assert np.linalg.norm((U * S) @ V - dense) <= 1e-13 * np.linalg.norm(dense)
