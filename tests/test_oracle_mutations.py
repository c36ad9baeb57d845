"""The pins are strong enough: each plausible mistake, planted in a
temporary copy of the oracle (on the CPU), makes at least one pin fail.

C oracle: a flipped sign, a dropped last term, a transposed B index, the
wrong leading dimension for A or C.  Split oracle: floor instead of
round-to-nearest, an off-by-one exponent, a dropped digit level, digits
combined with the wrong weight.  Low-rank oracle: see LOWRANK_MUTATIONS.

The bound helpers that set the GPU tolerances are covered the same way:
|C0| + |A||B| (oracle_gemm_absbound) without |C0|, without an |.| on C0, A
or B, or with C0 read at the wrong leading dimension; the split
recombination magnitude without |C|, with signed terms, unscaled terms or
the wrong level weight; the a-priori bound made looser (A's or B's rounding
term doubled, the dropped pairs counted twice) or too small (a term left
out); and the randomized SVD's flop count with the power iterations counted
once, the QRs without forming Q, the final V product or the n-row panels
miscounted."""
import ctypes
import importlib.util
import os
import subprocess
import sys
import types
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import PRESETS

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_DIR = os.path.join(os.path.dirname(HERE), "oracle")

C_MUTATIONS = {
    "sign": ("c[i] = c[i] + prod;", "c[i] = c[i] - prod;"),
    "dropped_term": ("for (int32_t p = 0; p < k; ++p) {\n            const double* a",
                     "for (int32_t p = 0; p < k - 1; ++p) {\n            const double* a"),
    "transposed_B": ("double b = B[(size_t)p + (size_t)j * (size_t)ldb];",
                     "double b = B[(size_t)j + (size_t)p * (size_t)ldb];"),
    "wrong_lda": ("const double* a = A + (size_t)p * (size_t)lda;", "const double* a = A + (size_t)p * (size_t)m;"),
    "wrong_ldc": ("double* c = C + (size_t)j * (size_t)ldc;", "double* c = C + (size_t)j * (size_t)m;"),
}


def build_mutant(tmp_path, old, new):
    src = open(os.path.join(ORACLE_DIR, "oracle_gemm.c")).read()
    assert src.count(old) == 1, old
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    "-o", str(so), str(path), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    i32 = ctypes.c_int32
    L.oracle_gemm.argtypes = [i32, i32, i32, dp, i32, dp, i32, dp, i32]
    return L


def pins_pass_c(L) -> bool:
    """A compact run of the FP64 pins against library L."""
    dp = ctypes.POINTER(ctypes.c_double)
    rng = np.random.default_rng(0)

    def run(m, n, k, A, lda, B, ldb, C, ldc):
        a = np.ascontiguousarray(A.ravel(order="F"))
        b = np.ascontiguousarray(B.ravel(order="F"))
        c = np.ascontiguousarray(C.ravel(order="F")).copy()
        L.oracle_gemm(m, n, k, a.ctypes.data_as(dp), lda, b.ctypes.data_as(dp), ldb, c.ctypes.data_as(dp), ldc)
        return c.reshape(C.shape, order="F")

    for m, n, k in [(5, 4, 3), (17, 5, 33)]:
        pad = 2
        A = np.zeros((m + pad, k))
        A[:m] = rng.integers(-8, 9, (m, k))
        B = np.zeros((k + pad, n))
        B[:k] = rng.integers(-8, 9, (k, n))
        C = np.zeros((m + pad, n))
        C[:m] = rng.integers(-100, 100, (m, n))
        out = run(m, n, k, A, m + pad, B, k + pad, C, m + pad)
        exact = C[:m] + A[:m] @ B[:k]
        if not np.array_equal(out[:m], exact) or not np.array_equal(out[m:], C[m:]):
            return False
    return True


def test_unmutated_oracle_passes():
    assert pins_pass_c(oracle.lib())


@pytest.mark.parametrize("name", sorted(C_MUTATIONS))
def test_c_mutation_is_caught(tmp_path, name):
    old, new = C_MUTATIONS[name]
    assert not pins_pass_c(build_mutant(tmp_path, old, new))


SPLIT_MUTATIONS = {
    "floor_not_rint": ("Z = np.rint(np.ldexp(", "Z = np.floor(np.ldexp("),
    "exponent_off_by_one": ("return np.where(mu == 0, 0, e).astype(np.int64)",
                            "return np.where(mu == 0, 0, e - 1).astype(np.int64)"),
    "dropped_level": ("        for L in sorted(levels):\n            scale",
                      "        for L in sorted(levels)[:-1]:\n            scale"),
    "wrong_weight": ("scale = (E[:, None] + F[None, :] - p.beta * L)", "scale = (E[:, None] + F[None, :] - p.beta * (L - 1))"),
}


def load_split_mutant(old, new) -> types.ModuleType:
    src = open(os.path.join(ORACLE_DIR, "split.py")).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("split_mutant")
    sys.modules["split_mutant"] = mod          # dataclasses look the module up
    try:
        exec(compile(src.replace(old, new), "split_mutant", "exec"), mod.__dict__)
    finally:
        del sys.modules["split_mutant"]
    return mod


def split_pins_pass(S) -> bool:
    p = PRESETS["bf16_s3"]
    rng = np.random.default_rng(1)
    # integer inputs: exact product
    m, n, k = 6, 5, p.kc + 9
    A = rng.integers(-8, 9, (m, k)).astype(np.float64)
    B = rng.integers(-8, 9, (k, n)).astype(np.float64)
    C = rng.integers(-50, 50, (m, n)).astype(np.float64)
    if not np.array_equal(S.split_gemm(A, B, C, p), C + A @ B):
        return False
    # digits reconstruct the correctly rounded value
    x = rng.standard_normal((3, 20)) * 10.0 ** rng.uniform(-3, 3, (3, 20))
    E = S.chunk_exponents(x, axis=1)
    for i in range(3):
        mu = max(abs(Fraction(v)) for v in x[i])
        if not (Fraction(2) ** (int(E[i]) - 1) <= mu < Fraction(2) ** int(E[i])):
            return False
    D = S.split_digits(x, E[:, None], p)
    rec = S.reconstruct(D, E[:, None], p)
    if np.any(np.abs(rec - x) > np.ldexp(1.0, (E[:, None] - p.beta * p.S - 1).astype(np.int32))):
        return False
    # a-priori bound on random data
    A = rng.standard_normal((4, 40))
    B = rng.standard_normal((40, 3))
    C = np.zeros((4, 3))
    out = S.split_gemm(A, B, C, p)
    bnd = oracle.apriori_bound(A, B, C, p)
    for i in range(4):
        for j in range(3):
            exact = sum(Fraction(A[i, q]) * Fraction(B[q, j]) for q in range(40))
            if abs(Fraction(out[i, j]) - exact) > Fraction(bnd[i, j]):
                return False
    return True


def test_unmutated_split_oracle_passes():
    import oracle.split as S
    assert split_pins_pass(S)


@pytest.mark.parametrize("name", sorted(SPLIT_MUTATIONS))
def test_split_mutation_is_caught(name):
    assert not split_pins_pass(load_split_mutant(*SPLIT_MUTATIONS[name]))


# Low-rank producer/consumer oracle (oracle/lowrank.py): an orthonormalisation
# left out, B formed from A^T, the trailing instead of the leading triplets
# kept, a power iteration without the transpose, the expansion without S, the
# rounded addition without S or with its core transposed.
LOWRANK_MUTATIONS = {
    "no_orthonormalisation": ("    Q = orth(A @ Omega)\n", "    Q = A @ Omega\n"),
    "B_from_A_transposed": ("    B = Q.T @ A\n", "    B = Q.T @ A.T\n"),
    "trailing_triplets": ("return Q @ Ut[:, :r], sigma[:r].copy(), Wt[:r, :].copy()",
                          "return Q @ Ut[:, -r:], sigma[-r:].copy(), Wt[-r:, :].copy()"),
    "power_without_transpose": ("        Qt = orth(A.T @ Q)\n", "        Qt = orth(A @ Q)\n"),
    "expand_unscaled": ("return D + (U * S[None, :]) @ V", "return D + U @ V"),
    "round_add_unscaled": ("Uc = np.hstack([U1 * S1[None, :], U2 * S2[None, :]])", "Uc = np.hstack([U1, U2])"),
    "round_add_core_transposed": ("np.linalg.svd(R1 @ R2.T)", "np.linalg.svd(R2 @ R1.T)"),
    "round_add_W_rows_for_columns": ("(Q2 @ Wt.T[:, :r]).T", "(Q2 @ Wt[:, :r]).T"),
    "round_add_V_blocks_swapped": ("Vc = np.vstack([V1, V2])", "Vc = np.vstack([V2, V1])"),
}


def load_lowrank_mutant(old, new) -> types.ModuleType:
    src = open(os.path.join(ORACLE_DIR, "lowrank.py")).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("lowrank_mutant")
    exec(compile(src.replace(old, new), "lowrank_mutant", "exec"), mod.__dict__)
    return mod


def lowrank_pins_pass(mod) -> bool:
    """Run the low-rank pins (test_oracle_lowrank) against module `mod`."""
    import importlib
    T = importlib.import_module("test_oracle_lowrank")
    cases = [(T.test_exact_rank_recovery, a) for a in [(60, 50, 5, 8, 0), (50, 80, 7, 7, 1), (33, 33, 1, 4, 0)]]
    cases += [(T.test_known_spectrum_truncation, (q,)) for q in (0, 2)]
    cases += [(T.test_range_finder_tail_bound, (q,)) for q in (0, 2)]
    cases += [(f, ()) for f in (T.test_eckart_young_full_sampling, T.test_power_iteration_sharpens,
                                T.test_orthonormal_factors, T.test_expand_integer_and_identity,
                                T.test_round_add_known_spectrum, T.test_round_add_exact_and_cancellation,
                                T.test_round_add_eckart_young_generic)]
    saved = T.L
    T.L = mod
    try:
        for f, args in cases:
            try:
                f(*args)
            except Exception:        # a failed assertion or a shape error: the pin caught it
                return False
    finally:
        T.L = saved
    return True


def test_unmutated_lowrank_oracle_passes():
    from oracle import lowrank
    assert lowrank_pins_pass(lowrank)


@pytest.mark.parametrize("name", sorted(LOWRANK_MUTATIONS))
def test_lowrank_mutation_is_caught(name):
    assert not lowrank_pins_pass(load_lowrank_mutant(*LOWRANK_MUTATIONS[name]))


# The bound helpers that set the GPU tolerances: |C0| + |A||B| (C oracle),
# the recombination magnitude and the a-priori bound (split oracle) and the
# randomized SVD's flop count.  Each planted mistake -- an |.| or a term left
# out, a scale or a weight wrong, a bound made looser -- fails a pin.
ABSBOUND_MUTATIONS = {
    "no_C0": ("= fabs(C0[(size_t)i", "= 0.0 * fabs(C0[(size_t)i"),
    "signed_C0": ("= fabs(C0[(size_t)i + (size_t)j * (size_t)ldc]);", "= (C0[(size_t)i + (size_t)j * (size_t)ldc]);"),
    "signed_A": ("+= fabs(A[(size_t)i + (size_t)p * (size_t)lda]) * b;", "+= A[(size_t)i + (size_t)p * (size_t)lda] * b;"),
    "signed_B": ("double b = fabs(B[(size_t)p", "double b = (B[(size_t)p"),
    "C0_wrong_ld": ("fabs(C0[(size_t)i + (size_t)j * (size_t)ldc])", "fabs(C0[(size_t)i + (size_t)j * (size_t)m])"),
}


def absbound_pins_pass(L) -> bool:
    import test_oracle_fp64 as T
    saved = oracle._lib
    oracle._lib = L
    try:
        T.test_absbound_exact_on_integers_and_dyadic_rationals()
        T.test_absbound_random_within_one_rounding_per_term()
    except AssertionError:
        return False
    finally:
        oracle._lib = saved
    return True


def test_unmutated_absbound_passes():
    assert absbound_pins_pass(oracle.lib())


@pytest.mark.parametrize("name", sorted(ABSBOUND_MUTATIONS))
def test_absbound_mutation_is_caught(tmp_path, name):
    L = build_mutant(tmp_path, *ABSBOUND_MUTATIONS[name])
    dp = ctypes.POINTER(ctypes.c_double)
    i32 = ctypes.c_int32
    L.oracle_gemm_absbound.argtypes = [i32, i32, i32, dp, i32, dp, i32, dp, i32, dp]
    L.oracle_gemm_absbound.restype = None
    assert not absbound_pins_pass(L)


SPLIT_HELPER_MUTATIONS = {
    "recomb_no_C": ("    mag = np.abs(np.asarray(C, dtype=np.float64)).copy()\n    nchunks",
                    "    mag = 0.0 * np.abs(np.asarray(C, dtype=np.float64))\n    nchunks"),
    "recomb_signed_terms": ("mag += np.ldexp(np.abs(P).astype(np.float64)", "mag += np.ldexp(P.astype(np.float64)"),
    "recomb_unscaled": ("mag += np.ldexp(np.abs(P).astype(np.float64), (E[:, None] + F[None, :] - p.beta * L).astype(np.int32))",
                        "mag += np.abs(P).astype(np.float64)"),
    "recomb_wrong_weight": ("- p.beta * L).astype(np.int32))\n    return mag", "- p.beta * (L - 1)).astype(np.int32))\n    return mag"),
    "apriori_loose_rounding": ("ea = np.ldexp(1.0, (E - p.beta * p.S - 1).astype(np.int32))",
                               "ea = np.ldexp(1.0, (E - p.beta * p.S).astype(np.int32))"),
    "apriori_loose_B_rounding": ("* eb[None, :]\n        dropped", "* 2 * eb[None, :]\n        dropped"),
    "apriori_dropped_twice": ("bound += (hi - lo) * dropped * sig", "bound += 2 * (hi - lo) * dropped * sig"),
    "apriori_without_A_rounding": ("        bound += ea[:, None] * absB.sum(axis=0)[None, :]\n", ""),
    "apriori_without_dropped": ("        if dropped:\n", "        if False:\n"),
}


def split_helper_pins_pass(S) -> bool:
    import test_oracle_split as T
    names = ("split_gemm", "apriori_bound", "recombination_magnitude", "split_digits", "chunk_exponents",
             "chunk_level_sums")
    saved = {n: getattr(oracle, n) for n in names}
    for n in names:
        setattr(oracle, n, getattr(S, n))
    try:
        for preset in ("bf16_s3", "fp16_s4"):
            T.test_recombination_magnitude_exact(preset)
            T.test_recombination_magnitude_wide_range(preset)
            T.test_apriori_bound_is_attained(preset)
            T.test_error_within_apriori_bound(preset)
    except AssertionError:
        return False
    finally:
        for n, f in saved.items():
            setattr(oracle, n, f)
    return True


def test_unmutated_split_helpers_pass():
    import oracle.split as S
    assert split_helper_pins_pass(S)


@pytest.mark.parametrize("name", sorted(SPLIT_HELPER_MUTATIONS))
def test_split_helper_mutation_is_caught(name):
    assert not split_helper_pins_pass(load_split_mutant(*SPLIT_HELPER_MUTATIONS[name]))


FLOPS_MUTATIONS = {
    "power_iteration_counted_once": ("gemm_a = 2.0 * m * n * l * (2 + 2 * q)", "gemm_a = 2.0 * m * n * l * (2 + q)"),
    "qr_without_forming_Q": ("qr = lambda rows: 2.0 * (2.0 * rows", "qr = lambda rows: 1.0 * (2.0 * rows"),
    "final_without_V": ("final = 2.0 * m * l * r + 2.0 * n * l * r", "final = 2.0 * m * l * r"),
    "n_panels_as_m": ("qrs = (1 + q) * qr(m) + (1 + q) * qr(n)", "qrs = (1 + q) * qr(m) + (1 + q) * qr(m)"),
}


def flops_pins_pass(mod) -> bool:
    import test_oracle_lowrank as T
    saved = T.L
    T.L = mod
    try:
        for args in [(30, 20, 6, 3, 0), (30, 20, 6, 3, 1), (41, 57, 9, 4, 2)]:
            T.test_lowrank_flops_against_counted_products(*args)
        T.test_lowrank_flops_literal_hand_count()
    except AssertionError:
        return False
    finally:
        T.L = saved
    return True


def test_unmutated_flops_pass():
    from oracle import lowrank
    assert flops_pins_pass(lowrank)


@pytest.mark.parametrize("name", sorted(FLOPS_MUTATIONS))
def test_flops_mutation_is_caught(name):
    assert not flops_pins_pass(load_lowrank_mutant(*FLOPS_MUTATIONS[name]))
