"""Seeded synthetic workloads for batched C_i += A_i * B_i.

This module only draws random shapes and values and lays them out in flat
buffers; it contains none of the multiplication's arithmetic, so both the
GPU path and the CPU oracle can be fed from it.

Shapes follow the low-rank setting of the paper: an (m, n, rank) block is
U S V (Eq. 1, Sec. 2), so its products are the tall-skinny "T-form"
C(b x r) += A(b x b) B(b x r) (dense block times a basis, e.g. the sampling
step of a randomized SVD) and the outer "O-form" C(b x b) += A(b x r) B(r x b)
(expanding U (S V) back to a dense block).  Values are N(0, 1) as in the
paper's experiments (Sec. 7) unless a workload says otherwise.  Every entry is
column-major; entries sit back to back in one flat buffer per operand unless
a workload says otherwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

FORM_T = 0   # C(b x r) += A(b x b) * B(b x r)
FORM_O = 1   # C(b x b) += A(b x r) * B(r x b)


def entry_shape(form: int, b: int, r: int):
    """(m, n, k) of one entry."""
    if form == FORM_T:
        return b, r, b
    if form == FORM_O:
        return b, b, r
    raise ValueError(f"unknown form {form}")


@dataclass
class Batch:
    """Flat operand buffers plus one descriptor row per entry.

    A, B, C are 1-D float64 tensors (host or device).  offA/offB/offC are
    element offsets of each entry's first element; m, n, k, lda, ldb, ldc the
    shapes.  `forms`, `bs`, `rs` record how each entry was drawn."""
    A: torch.Tensor
    B: torch.Tensor
    C: torch.Tensor
    m: np.ndarray
    n: np.ndarray
    k: np.ndarray
    lda: np.ndarray
    ldb: np.ndarray
    ldc: np.ndarray
    offA: np.ndarray
    offB: np.ndarray
    offC: np.ndarray
    forms: np.ndarray = field(default=None)
    bs: np.ndarray = field(default=None)
    rs: np.ndarray = field(default=None)
    name: str = ""

    def __len__(self):
        return len(self.m)

    def flops(self) -> float:
        return float(np.sum(2.0 * self.m.astype(np.float64) * self.n * self.k))

    def alg_bytes(self) -> float:
        """Each operand read once, C read and written once (8-byte elements)."""
        m, n, k = (x.astype(np.float64) for x in (self.m, self.n, self.k))
        return float(np.sum(8.0 * (m * k + k * n + 2.0 * m * n)))

    def to(self, device) -> "Batch":
        kw = dict(self.__dict__)
        kw["A"], kw["B"], kw["C"] = (t.to(device) for t in (self.A, self.B, self.C))
        return Batch(**kw)


def _fill(t: torch.Tensor, dist: str, gen: torch.Generator):
    if dist == "uniform":            # U[-1, 1]
        t.uniform_(-1.0, 1.0, generator=gen)
    elif dist == "normal":           # N(0, 1)
        t.normal_(0.0, 1.0, generator=gen)
    elif dist == "wide":             # 10^U(-4, 4) * N(0, 1)
        e = torch.empty_like(t).uniform_(-4.0, 4.0, generator=gen)
        t.normal_(0.0, 1.0, generator=gen)
        t.mul_(torch.pow(10.0, e))
    elif dist == "int8":             # integers in [-8, 8]: every sum is exact
        t.copy_(torch.randint(-8, 9, t.shape, generator=gen, device=t.device, dtype=torch.int64))
    else:
        raise ValueError(dist)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def uniform_batch(form: int, b: int, r: int, batch: int, *, dist: str = "normal",
                  seed: int = 0, device="cpu", pad: int = 0, name: str = "") -> Batch:
    """`batch` entries of one (form, b, r); ld = rows + pad.  A, B and C are
    drawn in that order from one generator seeded with `seed`."""
    m, n, k = entry_shape(form, b, r)
    lda, ldb, ldc = m + pad, k + pad, m + pad
    sa, sb, sc = lda * k, ldb * n, ldc * n
    g = _gen(seed, device)
    A = torch.empty(batch * sa, dtype=torch.float64, device=device)
    B = torch.empty(batch * sb, dtype=torch.float64, device=device)
    C = torch.empty(batch * sc, dtype=torch.float64, device=device)
    for t in (A, B, C):
        _fill(t, dist, g)
    ar = np.arange(batch, dtype=np.int64)
    full = lambda v: np.full(batch, v, dtype=np.int32)
    return Batch(A, B, C, full(m), full(n), full(k), full(lda), full(ldb), full(ldc),
                 ar * sa, ar * sb, ar * sc, forms=full(form), bs=full(b), rs=full(r),
                 name=name or f"{'TO'[form]}-b{b}-r{r}-x{batch}")


# --- the workload recipes ------------------------------------------------

def small_o_form(device="cpu") -> Batch:
    """O-form, 64 entries of C(256x256) += A(256x16) B(16x256); A, B, C drawn
    from U[-1, 1] in that order from a generator seeded with 0; contiguous
    column-major entries back to back."""
    return uniform_batch(FORM_O, 256, 16, 64, dist="uniform", seed=0, device=device,
                         name="O-b256-r16-x64")


UNIFORM_SWEEP_B = (256, 512, 1024)
UNIFORM_SWEEP_R = (16, 32, 64)
UNIFORM_SWEEP_BATCH = {256: 4096, 512: 1024, 1024: 256}


def uniform_sweep_groups():
    """The uniform-shape sweep: b in {256, 512, 1024} (batch 4096/1024/256),
    r in {16, 32, 64}, both forms, N(0, 1), seed 1000 + 100 form + 10 bi + ri.
    Yields (form, b, r, batch, seed)."""
    for form in (FORM_T, FORM_O):
        for bi, b in enumerate(UNIFORM_SWEEP_B):
            for ri, r in enumerate(UNIFORM_SWEEP_R):
                yield form, b, r, UNIFORM_SWEEP_BATCH[b], 1000 + 100 * form + 10 * bi + ri


def variable_shapes(count: int = 20000, seed: int = 3, bmin: int = 64, bmax: int = 2048,
                    ranks=(8, 16, 32, 64, 128)):
    """Shapes of the variable-size batch: b = round(exp(U(ln bmin, ln bmax))),
    r uniform over `ranks`, form T or O with probability 1/2 each."""
    rng = np.random.default_rng(seed)
    b = np.rint(np.exp(rng.uniform(math.log(bmin), math.log(bmax), count))).astype(np.int32)
    r = rng.choice(np.asarray(ranks, dtype=np.int32), count)
    form = rng.integers(0, 2, count).astype(np.int32)
    return form, b, r


def variable_batch(forms, bs, rs, *, seed: int = 3, device="cpu", pool_elems: int = None,
                   name: str = "variable") -> Batch:
    """Entries of the given shapes.  A and B are views into one shared N(0, 1)
    operand pool (read-only, so entries may overlap there); every entry has
    its own C, also N(0, 1).  The pool holds `pool_elems` doubles (default:
    just enough for the largest operand, times four)."""
    forms, bs, rs = (np.asarray(x, dtype=np.int32) for x in (forms, bs, rs))
    cnt = len(forms)
    m = np.where(forms == FORM_T, bs, bs).astype(np.int32)
    n = np.where(forms == FORM_T, rs, bs).astype(np.int32)
    k = np.where(forms == FORM_T, bs, rs).astype(np.int32)
    sizeA = m.astype(np.int64) * k
    sizeB = k.astype(np.int64) * n
    sizeC = m.astype(np.int64) * n
    need = int(max(sizeA.max(), sizeB.max()))
    if pool_elems is None:
        pool_elems = 4 * need
    pool_elems = max(pool_elems, need)
    rng = np.random.default_rng(seed + 7919)
    align = 32   # entry bases on 256-byte boundaries
    offA = (rng.integers(0, (pool_elems - sizeA) // align + 1) * align).astype(np.int64)
    offB = (rng.integers(0, (pool_elems - sizeB) // align + 1) * align).astype(np.int64)
    cstride = ((sizeC + align - 1) // align) * align
    offC = np.concatenate([[0], np.cumsum(cstride)[:-1]]).astype(np.int64)
    g = _gen(seed, device)
    pool = torch.empty(pool_elems, dtype=torch.float64, device=device)
    _fill(pool, "normal", g)
    C = torch.empty(int(cstride.sum()), dtype=torch.float64, device=device)
    _fill(C, "normal", g)
    return Batch(pool, pool, C, m, n, k, m.copy(), k.copy(), m.copy(), offA, offB, offC,
                 forms=forms, bs=bs, rs=rs, name=name)


def wide_range(form: int, batch: int = 2048, b: int = 1024, r: int = 64, device="cpu",
               seed: int = 4) -> Batch:
    """Split-precision workload: entries 10^U(-4,4) * N(0,1), b = 1024, r = 64."""
    return uniform_batch(form, b, r, batch, dist="wide", seed=seed, device=device,
                         name=f"wide-{'TO'[form]}-b{b}-r{r}-x{batch}")


def serving_requests(count: int, rate: float, seed: int = 5, max_products: int = 512,
                     bmin: int = 64, bmax: int = 2048, ranks=(8, 16, 32, 64, 128)):
    """Poisson request stream: arrival times (s), and per request the number
    of products (uniform 1..max_products) and their (form, b, r) as above."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    arrivals = np.cumsum(gaps)
    reqs = []
    for q in range(count):
        cnt = int(rng.integers(1, max_products + 1))
        b = np.rint(np.exp(rng.uniform(math.log(bmin), math.log(bmax), cnt))).astype(np.int32)
        r = rng.choice(np.asarray(ranks, dtype=np.int32), cnt)
        form = rng.integers(0, 2, cnt).astype(np.int32)
        reqs.append((form, b, r))
    return arrivals, reqs


@dataclass
class LrBatch:
    """Batched low-rank chain inputs: per entry A_{V^T} (ra x k), B_U (k x rb),
    A_X (ra x ra), B_X (rb x rb) and the output G (ra x rb), each in its own
    flat buffer, entries back to back, leading dimensions = rows + pad."""
    bufs: dict
    offs: dict
    ra: np.ndarray
    rb: np.ndarray
    k: np.ndarray
    pad: int = 0

    def __len__(self):
        return len(self.ra)

    def flops_paper(self) -> float:
        """The paper's count, batch (4 r^3 + 2 r^2 b) for ra = rb = r (Sec. 7, GFLOPS equation)."""
        r = self.ra.astype(np.float64)
        return float(np.sum(4 * r ** 3 + 2 * r ** 2 * self.k))

    def to(self, device) -> "LrBatch":
        return LrBatch({key: t.to(device) for key, t in self.bufs.items()}, self.offs, self.ra, self.rb, self.k,
                       self.pad)


def lr_batch(batch: int, b: int, r: int, *, rb: int = None, seed: int = 0, device="cpu", pad: int = 0,
             dist: str = "normal") -> LrBatch:
    """`batch` low-rank chains with rank r (and rb, default r) and block size
    b, entries N(0,1) (the paper's experiments use normally distributed
    entries, Sec. 7), drawn in the order A_{V^T}, B_U, A_X, B_X from one
    generator seeded with `seed`."""
    rb = r if rb is None else rb
    shapes = {"AVT": (r, b), "BU": (b, rb), "AX": (r, r), "BX": (rb, rb), "G": (r, rb)}
    g = _gen(seed, device)
    bufs, offs = {}, {}
    for key, (rows, cols) in shapes.items():
        size = (rows + pad) * cols
        t = torch.empty(batch * size, dtype=torch.float64, device=device)
        if key == "G":
            t.zero_()
        else:
            _fill(t, dist, g)
        bufs[key] = t
        offs[key] = np.arange(batch, dtype=np.int64) * size
    full = lambda v: np.full(batch, v, dtype=np.int32)
    return LrBatch(bufs, offs, full(r), full(rb), full(b), pad)


# ---- dense blocks for the low-rank producers --------------------------------
# Sec. 2: low-rank blocks come from dense blocks whose singular values decay
# fast, as the off-diagonal (admissible) blocks of hierarchical matrices do.
# Stand-in: the Laplace kernel 1/|x - y| between two separated point clusters
# (x uniform in the unit cube, y in the unit cube shifted by `sep` along the
# first axis), evaluated element by element; no product is formed.

def kernel_blocks(count: int, m: int, n: int, *, seed: int = 7, sep: float = 2.0, device="cpu",
                  chunk: int = 64) -> torch.Tensor:
    """`count` dense m x n blocks A_e[i, j] = 1 / |x_i - y_j|, column-major and
    back to back (entry e at offset e m n, ld = m), float64."""
    g = _gen(seed, device)
    out = torch.empty(count * m * n, dtype=torch.float64, device=device)
    shift = torch.tensor([sep, 0.0, 0.0], dtype=torch.float64, device=device)
    for c0 in range(0, count, chunk):
        c = min(chunk, count - c0)
        x = torch.rand((c, m, 3), generator=g, dtype=torch.float64, device=device)
        y = torch.rand((c, n, 3), generator=g, dtype=torch.float64, device=device) + shift
        d = torch.cdist(y, x, compute_mode="donot_use_mm_for_euclid_dist")    # [c, n, m]: (j, i) -> j m + i
        out[c0 * m * n:(c0 + c) * m * n] = d.reciprocal_().reshape(-1)
    return out


def gaussian_test_matrix(n: int, l: int, *, seed: int = 8, device="cpu") -> torch.Tensor:
    """The randomized SVD's n x l test matrix Omega: N(0, 1), column-major
    (ld = n), drawn from its own seeded generator."""
    g = _gen(seed, device)
    return torch.randn(n * l, generator=g, dtype=torch.float64, device=device)
