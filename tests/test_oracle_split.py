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
  stays under the a-priori bound, and shrinks by about 2^-beta per digit.
"""
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
