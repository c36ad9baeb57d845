"""Pins for the split-precision oracle (oracle/split.py), each against
something other than the oracle itself:

* digits: exact rational rounding (Python fractions) of a * 2^(beta S - E),
  and the sequential round-to-nearest digit recursion written out with
  fractions -- both must give the same integer as the balanced digits;
* digit ranges, and exact representability of every digit in the tensor-core
  operand type (a round trip through torch's bf16/fp16);
* every level sum of a chunk fits an FP32 accumulator exactly (|P_L| <= 2^24);
* integer inputs whose digits are exact: the split product is the exact
  integer product;
* random wide-range inputs: the error against the exact product (fractions)
  stays under the a-priori bound, and shrinks by about 2^-beta per digit;
* the a-priori bound from above: inputs that make every part of it tight at
  once (half-unit rounding ties, dropped digit pairs at their largest) reach
  it to within 0.1 %;
* the recombination magnitude (the tolerance of the GPU comparisons): equal
  to |C0| + sum |2^(E+F-beta L) P_L| written out with integer digits and
  fractions (bitwise on integer inputs, within gamma_n on wide-range ones).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from oracle import PRESETS, SplitParams


def rn_even_fraction(q: Fraction) -> int:
    fl = q.numerator // q.denominator
    rem = q - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        return fl + 1
    return fl


def sequential_digits(x: float, E: int, p: SplitParams):
    """Digits by the recursion d_s = RN(r_{s-1} 2^beta), r_s = r_{s-1} 2^beta - d_s,
    r_0 = x / 2^E, in exact arithmetic."""
    r = Fraction(x) / Fraction(2) ** E
    out = []
    for _ in range(p.S):
        v = r * 2 ** p.beta
        d = rn_even_fraction(v)
        out.append(d)
        r = v - d
    return out


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_digits_against_exact_rounding(name):
    p = PRESETS[name]
    rng = np.random.default_rng(7)
    x = rng.standard_normal((6, 40)) * 10.0 ** rng.uniform(-4, 4, (6, 40))
    x[0, :5] = [0.0, -0.0, 1.0, -0.5, 2.0 ** -1074]      # zero, powers of two, subnormal
    x[1, :] = 0.0                                          # an all-zero row
    x[2, 3] = 1.0 - 2.0 ** -53                             # rounds up to the top digit
    E = oracle.chunk_exponents(x, axis=1)
    assert E[1] == 0
    D = oracle.split_digits(x, E[:, None], p)
    base, half = 2 ** p.beta, 2 ** (p.beta - 1)
    assert np.all(np.abs(D[0]) <= base)
    assert np.all((D[1:] >= -half) & (D[1:] < half))
    for i in range(x.shape[0]):
        mu = max(abs(Fraction(v)) for v in x[i])
        if mu:
            assert Fraction(2) ** (E[i] - 1) <= mu < Fraction(2) ** E[i]
        for j in range(x.shape[1]):
            Z = rn_even_fraction(Fraction(x[i, j]) * Fraction(2) ** (p.beta * p.S - int(E[i])))
            val = 0
            for s in range(p.S):
                val = val * base + int(D[s, i, j])
            assert val == Z
            seq = sequential_digits(float(x[i, j]), int(E[i]), p)
            sval = 0
            for d in seq:
                sval = sval * base + d
            assert sval == Z            # the recursion reaches the same rounded integer
    rec = oracle.reconstruct(D, E[:, None], p)
    err = np.abs(rec - x)
    assert np.all(err <= np.ldexp(1.0, (E[:, None] - p.beta * p.S - 1).astype(np.int32)))


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_digits_exact_in_operand_type(name):
    p = PRESETS[name]
    lim = 2 ** p.beta
    d = torch.arange(-lim, lim + 1, dtype=torch.float64)
    dt = torch.bfloat16 if p.fmt == "bf16" else torch.float16
    assert torch.equal(d.to(dt).to(torch.float64), d)


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_level_sums_fit_fp32(name):
    p = PRESETS[name]
    for L in p.levels():
        assert oracle.level_bound(p, L) <= 2 ** 24
    # attain the largest digits: every element of A and B just below its row /
    # column maximum; level sums are integers in FP32's exact range.
    k = p.kc
    A = np.full((4, k), 1.0 - 2.0 ** -40)
    B = np.full((k, 3), -(1.0 - 2.0 ** -40))
    E, F, levels = oracle.chunk_level_sums(A, B, p, 0)
    for L, P in levels.items():
        assert np.all(np.abs(P) <= 2 ** 24)
        assert np.all(P.astype(np.float32).astype(np.int64) == P)


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_integer_inputs_exact(name):
    p = PRESETS[name]
    rng = np.random.default_rng(8)
    m, n, k = 9, 7, 3 * p.kc + 5          # several chunks and a ragged one
    A = rng.integers(-8, 9, (m, k)).astype(np.float64)
    B = rng.integers(-8, 9, (k, n)).astype(np.float64)
    C = rng.integers(-1000, 1000, (m, n)).astype(np.float64)
    out = oracle.split_gemm(A, B, C, p)
    exact = C.astype(np.int64) + A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(out, exact.astype(np.float64))


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_error_within_apriori_bound(name):
    p = PRESETS[name]
    rng = np.random.default_rng(9)
    m, n, k = 5, 4, p.kc + 17
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-4, 4, (m, k))
    B = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-4, 4, (k, n))
    C = rng.standard_normal((m, n))
    out = oracle.split_gemm(A, B, C, p)
    bnd = oracle.apriori_bound(A, B, C, p)
    for i in range(m):
        for j in range(n):
            exact = Fraction(C[i, j]) + sum(Fraction(A[i, q]) * Fraction(B[q, j]) for q in range(k))
            assert abs(Fraction(out[i, j]) - exact) <= Fraction(bnd[i, j])


def test_more_digits_more_accuracy():
    rng = np.random.default_rng(10)
    m, n, k = 32, 16, 256
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    C = np.zeros((m, n))
    ref = A @ B
    errs = []
    for S in (2, 3, 4, 5):
        p = SplitParams("bf16", 8, S, 128)
        out = oracle.split_gemm(A, B, C, p)
        errs.append(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    for a, b in zip(errs, errs[1:]):
        assert b < a * 2.0 ** -5          # each digit buys ~beta bits
    assert errs[-1] < 1e-11            # triangular truncation dominates at S = 5


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_element_sampler_matches_full_oracle(name):
    p = PRESETS[name]
    rng = np.random.default_rng(12)
    m, n, k = 7, 6, 2 * p.kc + 3
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-4, 4, (m, k))
    B = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-4, 4, (k, n))
    C = rng.standard_normal((m, n))
    full = oracle.split_gemm(A, B, C, p)
    I, J = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    I, J = I.ravel(), J.ravel()
    got = oracle.split_dot_samples(A[I, :], B[:, J].T, C[I, J], p)
    assert np.array_equal(got, full[I, J])
    mag = oracle.recombination_magnitude(A, B, C, p)
    assert np.all(mag >= np.abs(full) * (1 - 1e-12))


def exact_exponent(values) -> int:
    """E with 2^(E-1) <= max|x| < 2^E over `values` (0 when all are zero),
    found by comparing exact rationals with powers of two."""
    mu = max(abs(Fraction(v)) for v in values)
    if mu == 0:
        return 0
    E = 0
    while Fraction(2) ** E <= mu:
        E += 1
    while Fraction(2) ** (E - 1) > mu:
        E -= 1
    return E


def balanced_digits_int(Z: int, p: SplitParams):
    """Digits d_1..d_S of the integer Z, lowest first, each of d_2..d_S in
    [-2^(beta-1), 2^(beta-1)) (plain Python integers)."""
    base, half = 2 ** p.beta, 2 ** (p.beta - 1)
    out = [0] * p.S
    for s in range(p.S - 1, 0, -1):
        d = (Z + half) % base - half
        out[s] = d
        Z = (Z - d) // base
    out[0] = Z
    return out


def exact_level_terms(A, B, C, p: SplitParams):
    """Every term the recombination adds, as exact rationals: for each chunk
    and level L, 2^(E_i + F_j - beta L) P_L[i, j] with P_L the exact integer
    sum of d_s e_t over the chunk and the level's kept pairs.  Written from
    the definition with Python integers and fractions only."""
    m, k = A.shape
    n = B.shape[1]
    terms = [[[] for _ in range(n)] for _ in range(m)]
    kept = p.kept_pairs()
    for lo in range(0, k, p.kc):
        hi = min(lo + p.kc, k)
        E = [exact_exponent(A[i, lo:hi]) for i in range(m)]
        F = [exact_exponent(B[lo:hi, j]) for j in range(n)]
        DA = [[balanced_digits_int(rn_even_fraction(Fraction(A[i, q]) * Fraction(2) ** (p.beta * p.S - E[i])), p)
               for q in range(lo, hi)] for i in range(m)]
        DB = [[balanced_digits_int(rn_even_fraction(Fraction(B[q, j]) * Fraction(2) ** (p.beta * p.S - F[j])), p)
               for q in range(lo, hi)] for j in range(n)]
        for i in range(m):
            for j in range(n):
                PL = {}
                for q in range(hi - lo):
                    for s, t in kept:
                        PL[s + t] = PL.get(s + t, 0) + DA[i][q][s - 1] * DB[j][q][t - 1]
                for L, P in PL.items():
                    terms[i][j].append(Fraction(P) * Fraction(2) ** (E[i] + F[j] - p.beta * L))
    return terms


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_recombination_magnitude_exact(name):
    # recombination_magnitude is the tolerance of every split-precision GPU
    # comparison (the GPU adds the same exact terms in another grouping), so
    # it is pinned to |C0| + sum |2^(E+F-beta L) P_L| written out independently
    # with integer digits and fractions.  Small integer inputs with mixed
    # signs keep every term an integer below 2^53, so the binary64 sum in the
    # helper is exact and must match bitwise; some level sums are negative.
    p = PRESETS[name]
    rng = np.random.default_rng(31)
    m, n, k = 4, 3, p.kc + 7
    A = rng.integers(-9, 10, (m, k)).astype(np.float64)
    B = rng.integers(-9, 10, (k, n)).astype(np.float64)
    C = rng.integers(-500, 501, (m, n)).astype(np.float64)
    C[0, 0] = -777.0
    terms = exact_level_terms(A, B, C, p)
    assert any(t < 0 for row in terms for cell in row for t in cell)
    got = oracle.recombination_magnitude(A, B, C, p)
    for i in range(m):
        for j in range(n):
            exact = abs(Fraction(C[i, j])) + sum(abs(t) for t in terms[i][j])
            assert Fraction(got[i, j]) == exact, (i, j)


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_recombination_magnitude_wide_range(name):
    # Wide-range inputs (10^U(-4,4) N(0,1)): the terms are exact rationals of
    # many binades, so the helper's binary64 sum of n nonnegative terms lies
    # within gamma_n of the exact sum, from either side.
    p = PRESETS[name]
    rng = np.random.default_rng(32)
    m, n, k = 3, 2, 2 * p.kc + 5
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-4, 4, (m, k))
    B = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-4, 4, (k, n))
    C = rng.standard_normal((m, n))
    terms = exact_level_terms(A, B, C, p)
    got = oracle.recombination_magnitude(A, B, C, p)
    for i in range(m):
        for j in range(n):
            exact = abs(Fraction(C[i, j])) + sum(abs(t) for t in terms[i][j])
            g = Fraction(oracle.gamma(len(terms[i][j]) + 1))
            assert abs(Fraction(got[i, j]) - exact) <= g * exact


def worst_case_value(p: SplitParams, lead: int, E: int) -> float:
    """A value whose rounding to beta*S fractional bits below 2^E loses the
    most (exactly half a unit: a tie that rounds toward zero) and whose digits
    d_2..d_S all sit at -2^(beta-1), the largest magnitude the bound allows:
    (Z + 1/2) 2^(E - beta S) with Z = lead 2^(beta (S-1)) - 2^(beta-1) sum_s 2^(beta s)."""
    half = 2 ** (p.beta - 1)
    Z = lead * 2 ** (p.beta * (p.S - 1)) - half * sum(2 ** (p.beta * s) for s in range(p.S - 1))
    assert Z % 2 == 0                      # the tie rounds to Z itself
    return math.ldexp(Z + 0.5, E - p.beta * p.S)


@pytest.mark.parametrize("name", sorted(PRESETS))
def test_apriori_bound_is_attained(name):
    # The a-priori bound is pinned from above: on inputs built to make every
    # part of it tight at once -- each operand rounded by exactly half a unit
    # in the same direction, every dropped digit pair at its largest product
    # with the sign that adds to that rounding loss -- the measured error of
    # the split product against the exact product (fractions) reaches the
    # bound to within a tiny fraction.  A bound looser by any constant factor
    # fails this test; one that is too small fails test_error_within_apriori_bound.
    p = PRESETS[name]
    lead = 3 * 2 ** (p.beta - 2)           # 0.75 of the top digit's range
    a = worst_case_value(p, lead, 3)
    b = worst_case_value(p, lead + 1, -2)
    m, n, k = 2, 3, p.kc + p.kc // 2       # a full chunk and a partial one
    A = np.full((m, k), a)
    B = np.full((k, n), b)
    C = np.zeros((m, n))
    D = oracle.split_digits(np.array([[a]]), np.array([[3]]), p)
    assert all(int(D[s, 0, 0]) == -2 ** (p.beta - 1) for s in range(1, p.S))
    out = oracle.split_gemm(A, B, C, p)
    bnd = oracle.apriori_bound(A, B, C, p)
    exact = k * Fraction(a) * Fraction(b)
    for i in range(m):
        for j in range(n):
            err = abs(Fraction(out[i, j]) - exact)
            assert err <= Fraction(bnd[i, j])
            assert err >= Fraction(bnd[i, j]) * Fraction(999, 1000), (float(err), bnd[i, j])
