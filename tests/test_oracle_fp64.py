"""Pins for the FP64 oracle (oracle/oracle_gemm.c), each against something
other than the oracle itself:

* exact rational arithmetic (Python fractions) on every m, n, k in 1..6 with
  random leading-dimension padding: the oracle must lie within Higham's
  forward-error bound gamma_{k+1} (|C0| + |A||B|) of the exact value, and the
  padding must be untouched;
* closed forms that are exact in binary64: A = I (C0 + B), a permutation
  (C0 + P B), an integer rank-1 product, integer-valued random inputs;
* Eq. 1's low-rank form U S V: (U S) V against U (S V) through the oracle,
  within twice the bound;
* a library routine: numpy's matmul within the bound;
* the bound helper |C0| + |A||B| (the element-wise tolerance of the GPU
  comparisons): bitwise equal to the exact rational value on integer and
  dyadic inputs with mixed signs and ld padding, within gamma_{2k+1} of it on
  random inputs.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def run(m, n, k, A, lda, B, ldb, C, ldc):
    A = np.ascontiguousarray(A.ravel(order="F"))
    B = np.ascontiguousarray(B.ravel(order="F"))
    Cf = np.ascontiguousarray(C.ravel(order="F")).copy()
    oracle.gemm(m, n, k, A, 0, lda, B, 0, ldb, Cf, 0, ldc)
    return Cf.reshape(C.shape, order="F")


def padded(rng, rows, cols, pad, fill):
    X = np.full((rows + pad, cols), fill)
    X[:rows, :] = rng.standard_normal((rows, cols))
    return X


def test_exact_rational_all_small_shapes():
    rng = np.random.default_rng(11)
    u = 2.0 ** -53
    for m in range(1, 7):
        for n in range(1, 7):
            for k in range(1, 7):
                pa, pb, pc = rng.integers(0, 3, 3)
                A = padded(rng, m, k, pa, 7.5)
                B = padded(rng, k, n, pb, -3.25)
                C = padded(rng, m, n, pc, 1e300)
                out = run(m, n, k, A, m + pa, B, k + pb, C, m + pc)
                # untouched padding
                assert np.array_equal(out[m:, :], C[m:, :])
                g = (k + 1) * u / (1 - (k + 1) * u)
                for i in range(m):
                    for j in range(n):
                        exact = Fraction(C[i, j]) + sum(Fraction(A[i, p]) * Fraction(B[p, j])
                                                        for p in range(k))
                        mag = abs(C[i, j]) + sum(abs(A[i, p] * B[p, j]) for p in range(k))
                        err = abs(Fraction(out[i, j]) - exact)
                        assert err <= Fraction(g * mag * (1 + 4 * u)), (m, n, k, i, j)


def test_identity_and_permutation_exact():
    rng = np.random.default_rng(1)
    for b, r in [(1, 1), (7, 3), (64, 16), (37, 9)]:
        B = rng.standard_normal((b, r))
        C = rng.standard_normal((b, r))
        out = run(b, r, b, np.eye(b), b, B, b, C, b)
        assert np.array_equal(out, C + B)
        perm = rng.permutation(b)
        P = np.zeros((b, b))
        P[np.arange(b), perm] = 1.0
        out = run(b, r, b, P, b, B, b, C, b)
        assert np.array_equal(out, C + B[perm, :])


def test_integer_rank1_closed_form():
    # A_ip = (i+1)(p+1), B_pj = (j+1): C_ij = (i+1)(j+1) k(k+1)/2 exactly.
    for m, n, k in [(5, 4, 3), (64, 16, 64), (33, 2, 17), (8, 64, 8)]:
        i = np.arange(m)[:, None] + 1.0
        p = np.arange(k)[None, :] + 1.0
        A = i * p
        B = np.tile(np.arange(n)[None, :] + 1.0, (k, 1))
        out = run(m, n, k, A, m, B, k, np.zeros((m, n)), m)
        expect = (np.arange(m)[:, None] + 1.0) * (np.arange(n)[None, :] + 1.0) * (k * (k + 1) / 2)
        assert np.array_equal(out, expect)


def test_integer_valued_random_exact():
    # entries in [-8, 8], |C0| <= 2^20: every partial sum is an integer below
    # 2^53, so every summation order gives the exact integer result.
    rng = np.random.default_rng(5)
    for m, n, k in [(17, 5, 33), (64, 64, 16), (3, 40, 128)]:
        A = rng.integers(-8, 9, (m, k)).astype(np.float64)
        B = rng.integers(-8, 9, (k, n)).astype(np.float64)
        C = rng.integers(-2 ** 20, 2 ** 20, (m, n)).astype(np.float64)
        out = run(m, n, k, A, m, B, k, C, m)
        exact = C.astype(np.int64) + A.astype(np.int64) @ B.astype(np.int64)
        assert np.array_equal(out, exact.astype(np.float64))


def bound(A, B, C, k):
    u = 2.0 ** -53
    return oracle.gamma(k + 1) * (np.abs(C) + np.abs(A) @ np.abs(B)) * (1 + 4 * u)


def test_matches_library_matmul_within_bound():
    rng = np.random.default_rng(2)
    for m, n, k in [(256, 16, 256), (64, 64, 16), (100, 7, 300)]:
        A = rng.standard_normal((m, k))
        B = rng.standard_normal((k, n))
        C = rng.standard_normal((m, n))
        out = run(m, n, k, A, m, B, k, C, m)
        ref = C + A @ B
        # both are within gamma_{k+1} of the exact result
        assert np.all(np.abs(out - ref) <= 2 * bound(A, B, C, k))


def test_low_rank_associativity_eq1():
    # Eq. 1: a block is U S V.  Expanding (U S) V and U (S V) through the
    # oracle must agree within the two products' rounding bounds.
    rng = np.random.default_rng(3)
    for b, r in [(64, 8), (128, 16), (33, 5)]:
        U = rng.standard_normal((b, r))
        S = np.diag(rng.uniform(0.5, 2.0, r)) + 0.1 * rng.standard_normal((r, r))
        V = rng.standard_normal((r, b))
        US = run(b, r, r, U, b, S, r, np.zeros((b, r)), b)
        SV = run(r, b, r, S, r, V, r, np.zeros((r, b)), r)
        left = run(b, b, r, US, b, V, r, np.zeros((b, b)), b)
        right = run(b, b, r, U, b, SV, r, np.zeros((b, b)), b)
        g = oracle.gamma(2 * r + 2)
        mag = np.abs(U) @ np.abs(S) @ np.abs(V)
        assert np.all(np.abs(left - right) <= 2 * g * mag)


@pytest.mark.parametrize("nthreads", [1, 3])
def test_batch_entry_points_agree(nthreads):
    rng = np.random.default_rng(4)
    shapes = [(5, 3, 7), (16, 16, 4), (9, 1, 12)]
    entries, refs = [], []
    for m, n, k in shapes:
        A = rng.standard_normal(m * k)
        B = rng.standard_normal(k * n)
        C = rng.standard_normal(m * n)
        ref = C.copy()
        oracle.gemm(m, n, k, A, 0, m, B, 0, k, ref, 0, m)
        entries.append(dict(A=A, B=B, C=C, m=m, n=n, k=k, lda=m, ldb=k, ldc=m))
        refs.append(ref)
    used = oracle.gemm_batch(entries, nthreads=nthreads)
    assert used >= 1
    for e, ref in zip(entries, refs):
        assert np.array_equal(e["C"], ref)
    # element sampler: same summation order, so bitwise equal
    m, n, k = shapes[0]
    A = entries[0]["A"].reshape(k, m).T
    B = entries[0]["B"].reshape(n, k).T
    c0 = rng.standard_normal(m * n)
    full = c0.copy()
    oracle.gemm(m, n, k, entries[0]["A"], 0, m, entries[0]["B"], 0, k, full, 0, m)
    I, J = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    I, J = I.ravel(), J.ravel()
    out = oracle.gemm_elements(A[I, :], B[:, J].T, c0.reshape(n, m).T[I, J])
    assert np.array_equal(out, full.reshape(n, m).T[I, J])


def absbound_exact(m, n, k, A, B, C):
    """|C0| + |A| |B| in exact rational arithmetic (Python fractions)."""
    out = np.empty((m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            out[i, j] = abs(Fraction(C[i, j])) + sum(abs(Fraction(A[i, p])) * abs(Fraction(B[p, j]))
                                                     for p in range(k))
    return out


def test_absbound_exact_on_integers_and_dyadic_rationals():
    # oracle_gemm_absbound sets the element-wise tolerance of every FP64 GPU
    # comparison, so it is pinned to |C0| + sum_p |a_ip| |b_pj| itself: on
    # integer and small dyadic-rational inputs every product and partial sum
    # is exact in binary64, so the helper must equal the exact value bitwise.
    # Signs are mixed (an |.| left out changes the value), the padding rows
    # hold huge values (reading them would show), and C0 is nonzero.
    rng = np.random.default_rng(21)
    for m, n, k, scale in [(1, 1, 1, 1.0), (5, 4, 3, 1.0), (17, 6, 33, 0.25), (9, 13, 70, 0.125)]:
        pa, pb, pc = rng.integers(1, 4, 3)
        A = np.full((m + pa, k), 1e300)
        B = np.full((k + pb, n), -1e300)
        C = np.full((m + pc, n), 1e300)
        A[:m] = rng.integers(-8, 9, (m, k)) * scale
        B[:k] = rng.integers(-8, 9, (k, n)) * scale
        C[:m] = rng.integers(-1000, 1001, (m, n)) * scale
        Af, Bf, Cf = (np.ascontiguousarray(X.ravel(order="F")) for X in (A, B, C))
        got = oracle.absbound(m, n, k, Af, 0, m + pa, Bf, 0, k + pb, Cf, 0, m + pc)
        exact = absbound_exact(m, n, k, A, B, C)
        assert got.shape == (m, n)
        for i in range(m):
            for j in range(n):
                assert Fraction(got[i, j]) == exact[i, j], (m, n, k, i, j)


def test_absbound_random_within_one_rounding_per_term():
    # Random binary64 inputs: the helper sums k + 1 nonnegative terms, so it is
    # within gamma_{2k+1} (one rounding per product and per addition) of the
    # exact value from below and above; offsets into a larger buffer are used.
    rng = np.random.default_rng(22)
    m, n, k = 7, 5, 40
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-3, 3, (m, k))
    B = rng.standard_normal((k, n))
    C = rng.standard_normal((m, n))
    Af = np.concatenate([np.zeros(11), A.ravel(order="F")])
    Bf = np.concatenate([np.zeros(5), B.ravel(order="F")])
    Cf = np.concatenate([np.zeros(3), C.ravel(order="F")])
    got = oracle.absbound(m, n, k, Af, 11, m, Bf, 5, k, Cf, 3, m)
    exact = absbound_exact(m, n, k, A, B, C)
    g = Fraction(oracle.gamma(2 * k + 1))
    for i in range(m):
        for j in range(n):
            assert abs(Fraction(got[i, j]) - exact[i, j]) <= g * exact[i, j]
