"""Split-precision (Ozaki-style) oracle for C += A @ B.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
CPU-baseline leg of the benchmark; never by the library.

The paper computes every product in binary64 (Sec. 7) and has no mixed
precision; the split path follows the error-free splitting of Ozaki, Ogita,
Oishi and Rump (Numer. Algorithms 59, 2012): each binary64 operand is cut into
S small-integer "digit" matrices that a BF16/FP16 tensor core multiplies
exactly with FP32 accumulation, and the digit products are recombined in
binary64.  The concrete choices (exponent per row/column per k-chunk, the
rounding to beta*S fractional bits, balanced digits, which digit pairs are
kept, chunk length) are this library's reading of that scheme and are stated
below; the GPU path implements the same definition independently.

Definition, for one k-chunk c (columns c*kc .. of A, the same rows of B):

1. Scale.  For row i of A, mu = max_p |a_ip| over the chunk.  If mu == 0 the
   row's digits are all zero.  Otherwise E_ic is the integer with
   2^(E_ic - 1) <= mu < 2^E_ic, so |a_ip| / 2^E_ic < 1.  Columns of B get F_jc
   the same way over the chunk's rows.
2. Round once.  Z = RN_even(a * 2^(beta*S - E)) is an integer, |Z| <= 2^(beta*S).
3. Balanced digits, lowest first: for s = S .. 2,
       d_s = ((Z + 2^(beta-1)) mod 2^beta) - 2^(beta-1)   in [-2^(beta-1), 2^(beta-1))
       Z   = (Z - d_s) / 2^beta
   and d_1 = the remaining Z, |d_1| <= 2^beta.  Then
       a ~= 2^E * sum_s d_s 2^(-beta*s),  with error <= 2^(E - beta*S - 1).
   Every digit is an integer with at most beta+1 significant bits, exact in
   BF16 (beta = 8) and FP16 (beta = 9).
4. Digit products.  P_st = D_s(A) @ D_t(B) over the chunk, for the kept pairs
   (s, t): "triangular" keeps s + t <= S + 1, "full" keeps all S*S.  Pairs of
   one level L = s + t share the scale 2^(E_i + F_j - beta*L) and are summed
   as integers: P_L = sum_{s+t=L} P_st.  kc is chosen so |P_L| <= 2^24, so an
   FP32 accumulator holds every partial sum exactly.
5. Recombine in binary64: for each chunk in k order and each level in
   increasing L,  C_ij <- C_ij + 2^(E_ic + F_jc - beta*L) * P_L[i, j].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class SplitParams:
    """Digit width beta, digit count S, k-chunk length kc, kept pairs."""
    fmt: str          # "bf16" or "fp16": the tensor-core operand type
    beta: int
    S: int
    kc: int
    pairs: str = "triangular"

    def kept_pairs(self):
        out = []
        for s in range(1, self.S + 1):
            for t in range(1, self.S + 1):
                if self.pairs == "full" or s + t <= self.S + 1:
                    out.append((s, t))
        return out

    def levels(self):
        return sorted({s + t for s, t in self.kept_pairs()})


# The four configurations of the split path (BF16/FP16 x 3/4 digits).  The
# chunk lengths keep every level sum within 2^24 (see level_bound below).
PRESETS = {
    "bf16_s3": SplitParams("bf16", 8, 3, 64),
    "bf16_s4": SplitParams("bf16", 8, 4, 64),
    "fp16_s3": SplitParams("fp16", 9, 3, 32),
    "fp16_s4": SplitParams("fp16", 9, 4, 32),
}


def level_bound(p: SplitParams, L: int) -> int:
    """Largest |P_L| one chunk can produce: kc * sum over the level's pairs of
    max|d_s| * max|e_t|, with max|d_1| = 2^beta and max|d_s| = 2^(beta-1), s>1."""
    def dmax(s):
        return 2 ** p.beta if s == 1 else 2 ** (p.beta - 1)
    return p.kc * sum(dmax(s) * dmax(t) for s, t in p.kept_pairs() if s + t == L)


def chunk_exponents(x: np.ndarray, axis: int) -> np.ndarray:
    """E with 2^(E-1) <= max|x| < 2^E along `axis` (0 where the max is 0).
    numpy's frexp returns exactly this exponent (mantissa in [0.5, 1))."""
    mu = np.max(np.abs(x), axis=axis)
    _, e = np.frexp(mu)
    return np.where(mu == 0, 0, e).astype(np.int64)


def split_digits(x: np.ndarray, E: np.ndarray, p: SplitParams) -> np.ndarray:
    """Digits of x (2-D) given per-element exponents E (broadcastable to x).
    Returns int64 array of shape (S,) + x.shape with x ~= 2^E sum_s d_s 2^(-beta s)."""
    shift = p.beta * p.S - E
    # ldexp by an integer power of two is exact (results that fall into the
    # subnormal range are < 2^-1022 and round to 0 below either way); rint is
    # round-half-to-even, so Z is the single correctly rounded integer.
    Z = np.rint(np.ldexp(x, shift.astype(np.int32) if np.ndim(shift) else int(shift)))
    Z = Z.astype(np.int64)
    base = 1 << p.beta
    half = 1 << (p.beta - 1)
    digits = np.zeros((p.S,) + x.shape, dtype=np.int64)
    for s in range(p.S, 1, -1):
        d = np.mod(Z + half, base) - half
        digits[s - 1] = d
        Z = (Z - d) // base
    digits[0] = Z
    return digits


def reconstruct(digits: np.ndarray, E: np.ndarray, p: SplitParams) -> np.ndarray:
    """sum_s d_s 2^(E - beta s) in binary64 (exact: the integer sum has at
    most beta*S+1 bits)."""
    Z = np.zeros(digits.shape[1:], dtype=np.int64)
    for s in range(p.S):
        Z = Z * (1 << p.beta) + digits[s]
    return np.ldexp(Z.astype(np.float64), (E - p.beta * p.S).astype(np.int32))


def chunk_level_sums(A: np.ndarray, B: np.ndarray, p: SplitParams, c: int):
    """For chunk c of A (m x k) @ B (k x n): (E (m,), F (n,), {L: P_L int64 (m, n)})."""
    k = A.shape[1]
    lo, hi = c * p.kc, min((c + 1) * p.kc, k)
    Ac, Bc = A[:, lo:hi], B[lo:hi, :]
    E = chunk_exponents(Ac, axis=1)
    F = chunk_exponents(Bc, axis=0)
    DA = split_digits(Ac, E[:, None], p)
    DB = split_digits(Bc, F[None, :], p)
    levels = {}
    for s, t in p.kept_pairs():
        P = DA[s - 1] @ DB[t - 1]          # int64 matmul: exact
        L = s + t
        levels[L] = levels.get(L, 0) + P
    return E, F, levels


def split_gemm(A: np.ndarray, B: np.ndarray, C: np.ndarray, p: SplitParams) -> np.ndarray:
    """Return C + (split-precision A @ B) as defined in the module docstring.
    A is m x k, B is k x n, C is m x n (any memory order), all float64."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.array(C, dtype=np.float64, copy=True)
    k = A.shape[1]
    nchunks = (k + p.kc - 1) // p.kc
    for c in range(nchunks):
        E, F, levels = chunk_level_sums(A, B, p, c)
        for L in sorted(levels):
            scale = (E[:, None] + F[None, :] - p.beta * L).astype(np.int32)
            out = out + np.ldexp(levels[L].astype(np.float64), scale)
    return out


def apriori_bound(A: np.ndarray, B: np.ndarray, C: np.ndarray, p: SplitParams) -> np.ndarray:
    """Elementwise bound on |split_gemm(A,B,C) - (C + A@B exactly)|.

    Per chunk, with a = ahat + da (|da| <= 2^(E-beta S-1)) and likewise b:
    |a b - ahat bhat| <= |da| |b| + |ahat| |db|, plus the dropped pairs
    (each |d_s e_t| <= 2^(2 beta - 2) for s, t >= 2) and the binary64
    recombination (one rounding per added term, bounded by gamma_n of the
    number of terms times the sum of their magnitudes plus |C|)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    n = B.shape[1]
    u = 2.0 ** -53
    bound = np.zeros((m, n))
    mag = np.abs(np.asarray(C, dtype=np.float64)).copy()
    nterms = 0
    nchunks = (k + p.kc - 1) // p.kc
    kept = set(p.kept_pairs())
    for c in range(nchunks):
        lo, hi = c * p.kc, min((c + 1) * p.kc, k)
        Ac, Bc = A[:, lo:hi], B[lo:hi, :]
        E = chunk_exponents(Ac, axis=1)
        F = chunk_exponents(Bc, axis=0)
        ea = np.ldexp(1.0, (E - p.beta * p.S - 1).astype(np.int32))   # max |da| per row
        eb = np.ldexp(1.0, (F - p.beta * p.S - 1).astype(np.int32))   # max |db| per column
        absA, absB = np.abs(Ac), np.abs(Bc)
        bound += ea[:, None] * absB.sum(axis=0)[None, :]
        bound += (absA + ea[:, None]).sum(axis=1)[:, None] * eb[None, :]
        dropped = 0.0
        for s in range(2, p.S + 1):
            for t in range(2, p.S + 1):
                if (s, t) not in kept:
                    dropped += 2.0 ** (-p.beta * (s + t) + 2 * p.beta - 2)
        if dropped:
            sig = np.ldexp(1.0, E.astype(np.int32))
            tau = np.ldexp(1.0, F.astype(np.int32))
            bound += (hi - lo) * dropped * sig[:, None] * tau[None, :]
        mag += (absA + ea[:, None]) @ (absB + eb[None, :])
        nterms += len(p.levels())
    g = nterms * u / (1 - nterms * u)
    return bound * (1 + 8 * u) + g * mag * (1 + 8 * u)


def split_dot_samples(arow: np.ndarray, bcol: np.ndarray, c0: np.ndarray, p: SplitParams) -> np.ndarray:
    """Selected outputs of split_gemm, one per sample: arow (q, k) holds row i
    of A, bcol (q, k) column j of B, c0 (q,) the old C value.  Row and column
    exponents depend only on that row and column, so each output follows the
    module definition exactly (same additions in the same order)."""
    arow = np.asarray(arow, dtype=np.float64)
    bcol = np.asarray(bcol, dtype=np.float64)
    out = np.array(c0, dtype=np.float64, copy=True)
    k = arow.shape[1]
    nchunks = (k + p.kc - 1) // p.kc
    for c in range(nchunks):
        lo, hi = c * p.kc, min((c + 1) * p.kc, k)
        Ar, Bc = arow[:, lo:hi], bcol[:, lo:hi]
        E = chunk_exponents(Ar, axis=1)
        F = chunk_exponents(Bc, axis=1)
        DA = split_digits(Ar, E[:, None], p)
        DB = split_digits(Bc, F[:, None], p)
        levels = {}
        for s, t in p.kept_pairs():
            P = np.sum(DA[s - 1] * DB[t - 1], axis=1)
            L = s + t
            levels[L] = levels.get(L, 0) + P
        for L in sorted(levels):
            out = out + np.ldexp(levels[L].astype(np.float64), (E + F - p.beta * L).astype(np.int32))
    return out


def recombination_magnitude(A: np.ndarray, B: np.ndarray, C: np.ndarray, p: SplitParams) -> np.ndarray:
    """|C| + sum over chunks and levels of |2^(E+F-beta L) P_L|: the size of
    everything the binary64 recombination adds, for rounding-error bounds of
    a recombination that adds the same exact terms in another grouping."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    mag = np.abs(np.asarray(C, dtype=np.float64)).copy()
    nchunks = (A.shape[1] + p.kc - 1) // p.kc
    for c in range(nchunks):
        E, F, levels = chunk_level_sums(A, B, p, c)
        for L, P in levels.items():
            mag += np.ldexp(np.abs(P).astype(np.float64), (E[:, None] + F[None, :] - p.beta * L).astype(np.int32))
    return mag
