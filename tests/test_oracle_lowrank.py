"""Pins for the low-rank producer/consumer oracle (oracle/lowrank.py), each
against something other than the oracle itself:

* exact recovery: a block of rank k <= l is reproduced to rounding error by
  the randomized SVD (range(A Omega) = range(A) with probability one);
* known spectrum: A = P diag(sigma) Q^T built from orthonormal P, Q and chosen
  sigma; the returned S is sigma's leading r values and U S V is the unique
  rank-r truncation P_r diag(sigma_r) Q_r^T;
* Eckart-Young with full sampling (l = n): the rank-r error is sigma_{r+1} in
  the spectral norm and the tail's root-sum-square in the Frobenius norm;
* Halko et al.'s tail bound for the range finder: with oversampling p >= 4,
  ||A - Q Q^T A|| <= (1 + 11 sqrt(k + p) sqrt(min(m, n))) sigma_{k+1} except
  with probability <= 6 p^-p; with q power iterations the same bound holds
  for the (2q+1)-th power of the error and sigma_{k+1}^(2q+1);
* orthonormal factors;
* expansion: exact on integer data, identity factors;
* rounded addition: two blocks built from disjoint columns of one
  orthonormal pair, so the singular values of the sum are known exactly; a
  sum whose rank fits is reproduced; X + (-X) gives zero;
* the flop count of the randomized SVD: its products against a count of the
  multiply-adds the oracle really performs, its QRs and the whole count
  against hand counts (Golub and Van Loan's Householder figures).
"""
import numpy as np
import pytest

from oracle import lowrank as L


def orthonormal(rng, rows, cols):
    Q, _ = np.linalg.qr(rng.standard_normal((rows, cols)))
    return Q


def known_spectrum(rng, m, n, sigma):
    P = orthonormal(rng, m, len(sigma))
    Q = orthonormal(rng, n, len(sigma))
    return P, Q, (P * sigma[None, :]) @ Q.T


def fro_rel(X, Y):
    return np.linalg.norm(X - Y) / np.linalg.norm(Y)


@pytest.mark.parametrize("m,n,k,l,q", [(60, 50, 5, 8, 0), (50, 80, 7, 7, 1), (128, 96, 16, 26, 2), (33, 33, 1, 4, 0)])
def test_exact_rank_recovery(m, n, k, l, q):
    rng = np.random.default_rng(m * 1000 + n)
    A = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
    U, S, V = L.rsvd(A, rng.standard_normal((n, l)), k, q)
    assert U.shape == (m, k) and S.shape == (k,) and V.shape == (k, n)
    assert fro_rel((U * S) @ V, A) < 1e-13


@pytest.mark.parametrize("q", [0, 1, 2])
def test_known_spectrum_truncation(q):
    rng = np.random.default_rng(11 + q)
    sigma = 10.0 ** (-0.5 * np.arange(8))          # exact rank 8 <= l
    P, Qm, A = known_spectrum(rng, 90, 70, sigma)
    r, l = 5, 12
    U, S, V = L.rsvd(A, rng.standard_normal((70, l)), r, q)
    assert np.all(np.abs(S - sigma[:r]) <= 1e-13 * sigma[0])
    assert np.all(np.diff(S) < 0)
    best = (P[:, :r] * sigma[:r]) @ Qm[:, :r].T
    assert np.linalg.norm((U * S) @ V - best) <= 1e-13 * np.linalg.norm(A)


def test_eckart_young_full_sampling():
    rng = np.random.default_rng(5)
    m, n = 80, 40
    sigma = np.linspace(4.0, 0.5, n)
    _, _, A = known_spectrum(rng, m, n, sigma)
    for r in (1, 7, 20):
        U, S, V = L.rsvd(A, rng.standard_normal((n, n)), r)
        E = A - (U * S) @ V
        assert abs(np.linalg.norm(E, 2) - sigma[r]) <= 1e-12 * sigma[0]
        assert abs(np.linalg.norm(E) - np.sqrt(np.sum(sigma[r:] ** 2))) <= 1e-12 * sigma[0]


@pytest.mark.parametrize("q", [0, 1, 2])
def test_range_finder_tail_bound(q):
    rng = np.random.default_rng(21)
    m, n, k, p = 200, 160, 10, 10
    sigma = 1.0 / (1.0 + np.arange(n))             # slow decay: the bound is not trivial
    _, _, A = known_spectrum(rng, m, n, sigma)
    Q = L.range_finder(A, rng.standard_normal((n, k + p)), q)
    err = np.linalg.norm(A - Q @ (Q.T @ A), 2)
    factor = 1 + 11 * np.sqrt(k + p) * np.sqrt(min(m, n))
    assert err <= factor ** (1.0 / (2 * q + 1)) * sigma[k] * (1 + 1e-12)
    assert err >= sigma[k + p] * (1 - 1e-12)        # no basis of k + p columns beats sigma_{k+p+1}
    # the truncated SVD adds at most sigma_{k+1} on top of the range error
    U, S, V = L.rsvd(A, rng.standard_normal((n, k + p)), k, q)
    assert np.linalg.norm(A - (U * S) @ V, 2) <= (factor ** (1.0 / (2 * q + 1)) + 1) * sigma[k]


def test_power_iteration_sharpens():
    rng = np.random.default_rng(8)
    m, n, k, p = 150, 150, 8, 6
    sigma = 1.0 / np.sqrt(1.0 + np.arange(n))
    _, _, A = known_spectrum(rng, m, n, sigma)
    Om = rng.standard_normal((n, k + p))
    errs = [np.linalg.norm(A - (lambda Q: Q @ (Q.T @ A))(L.range_finder(A, Om, q)), 2) for q in (0, 3)]
    assert errs[1] < 0.75 * errs[0]


def test_orthonormal_factors():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((120, 90))
    U, S, V = L.rsvd(A, rng.standard_normal((90, 30)), 20, 1)
    assert np.abs(U.T @ U - np.eye(20)).max() < 1e-14
    assert np.abs(V @ V.T - np.eye(20)).max() < 1e-14
    assert np.all(S > 0) and np.all(np.diff(S) <= 0)


def test_argument_checks():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((10, 8))
    with pytest.raises(ValueError):
        L.rsvd(A, rng.standard_normal((8, 9)), 3)       # l > min(m, n)
    with pytest.raises(ValueError):
        L.rsvd(A, rng.standard_normal((8, 4)), 5)       # r > l


def test_expand_integer_and_identity():
    rng = np.random.default_rng(2)
    m, n, r = 17, 13, 4
    U = rng.integers(-5, 6, (m, r)).astype(float)
    S = rng.integers(-3, 4, r).astype(float)
    V = rng.integers(-5, 6, (r, n)).astype(float)
    D = rng.integers(-100, 100, (m, n)).astype(float)
    exact = D.astype(np.int64) + (U.astype(np.int64) * S.astype(np.int64)) @ V.astype(np.int64)
    assert np.array_equal(L.lr_expand(U, S, V, D), exact.astype(float))
    X = rng.standard_normal((r, n))
    assert np.array_equal(L.lr_expand(np.eye(r), np.ones(r), X, np.zeros((r, n))), X)


def test_round_add_known_spectrum():
    rng = np.random.default_rng(31)
    m, n = 70, 60
    P, Qm = orthonormal(rng, m, 12), orthonormal(rng, n, 12)
    s1 = np.array([9.0, 5.0, 3.0, 1.0, 0.25, 0.1])
    s2 = np.array([7.0, 4.0, 2.0, 0.5, 0.2, 0.05])
    U1, V1 = P[:, :6], Qm[:, :6].T
    U2, V2 = P[:, 6:], Qm[:, 6:].T
    dense = (U1 * s1) @ V1 + (U2 * s2) @ V2
    allv = np.sort(np.concatenate([s1, s2]))[::-1]
    for r in (1, 4, 7, 12):
        U, S, V = L.lr_round_add(U1, s1, V1, U2, s2, V2, r)
        assert np.all(np.abs(S - allv[:r]) <= 1e-13 * allv[0])
        E = dense - (U * S) @ V
        tail = allv[r] if r < 12 else 0.0
        assert abs(np.linalg.norm(E, 2) - tail) <= 1e-13 * allv[0]


def test_round_add_exact_and_cancellation():
    rng = np.random.default_rng(32)
    m, n, r1, r2 = 64, 48, 5, 7
    U1, V1, S1 = rng.standard_normal((m, r1)), rng.standard_normal((r1, n)), rng.uniform(1, 2, r1)
    U2, V2, S2 = rng.standard_normal((m, r2)), rng.standard_normal((r2, n)), rng.uniform(1, 2, r2)
    dense = (U1 * S1) @ V1 + (U2 * S2) @ V2
    U, S, V = L.lr_round_add(U1, S1, V1, U2, S2, V2, r1 + r2)
    assert fro_rel((U * S) @ V, dense) < 1e-13
    U, S, V = L.lr_round_add(U1, S1, V1, U1, -S1, V1, 3)
    assert np.abs(S).max() <= 1e-13 * np.linalg.norm((U1 * S1) @ V1, 2)


def test_round_add_eckart_young_generic():
    """Generic (non-orthogonal) factors: the rank-r result is the best rank-r
    approximation of the dense sum (Eckart and Young), so its singular values
    are the sum's r leading ones and its Frobenius error is the norm of the
    rest -- both taken here from an SVD of the whole m x n sum, a route that
    shares nothing with the oracle's QR of the stacked bases."""
    rng = np.random.default_rng(33)
    m, n, r1, r2 = 80, 55, 6, 9
    U1, V1, S1 = rng.standard_normal((m, r1)), rng.standard_normal((r1, n)), np.logspace(0, -3, r1)
    U2, V2, S2 = rng.standard_normal((m, r2)), rng.standard_normal((r2, n)), np.logspace(-1, -4, r2)
    dense = (U1 * S1) @ V1 + (U2 * S2) @ V2
    sig = np.linalg.svd(dense, compute_uv=False)
    for r in (1, 5, 10, 15):
        U, S, V = L.lr_round_add(U1, S1, V1, U2, S2, V2, r)
        assert np.abs(S - sig[:r]).max() <= 1e-12 * sig[0]
        err = np.linalg.norm(dense - (U * S) @ V)
        assert abs(err - np.sqrt(np.sum(sig[r:] ** 2))) <= 1e-12 * sig[0]


class _CountingArray(np.ndarray):
    """ndarray that adds 2 m k n to a counter for every m x k by k x n
    matrix product taken with it (numpy's matmul ufunc), so the products the
    oracle's randomized SVD actually performs can be counted."""
    flops = 0

    def __array_ufunc__(self, ufunc, method, *inputs, **kw):
        raw = [np.asarray(x) if isinstance(x, _CountingArray) else x for x in inputs]
        if ufunc is np.matmul and method == "__call__":
            a, b = raw
            _CountingArray.flops += 2 * a.shape[0] * a.shape[1] * b.shape[-1]
        out = getattr(ufunc, method)(*raw, **kw)
        return out.view(_CountingArray) if isinstance(out, np.ndarray) else out


@pytest.mark.parametrize("m,n,l,r,q", [(30, 20, 6, 3, 0), (30, 20, 6, 3, 1), (41, 57, 9, 4, 2)])
def test_lowrank_flops_against_counted_products(m, n, l, r, q):
    # lowrank_flops is the throughput count of the randomized SVD.  Its product
    # part is pinned by counting the multiply-adds of the products the oracle
    # really takes (A Omega, q times A^T Q and A Q~, stage B's Q^T A, and
    # U = Q U~_r); the GPU also forms V by one n x l by l x r product.  The
    # QRs are counted by hand from Golub and Van Loan: Householder QR of a
    # rows x l panel is 2 l^2 (rows - l/3) flops and forming its thin Q as
    # much again; 1 + q panels of m rows and 1 + q of n rows.
    rng = np.random.default_rng(m + n + q)
    _CountingArray.flops = 0
    A = rng.standard_normal((m, n)).view(_CountingArray)
    Om = rng.standard_normal((n, l)).view(_CountingArray)
    L.rsvd(A, Om, r, q)
    counted = _CountingArray.flops
    assert counted == 2 * m * n * l * (2 + 2 * q) + 2 * m * l * r
    qr_hand = (1 + q) * 2 * (2 * l * l * (m - l / 3)) + (1 + q) * 2 * (2 * l * l * (n - l / 3))
    assert L.lowrank_flops(m, n, l, r, q) == pytest.approx(counted + 2 * n * l * r + qr_hand, rel=1e-15)


def test_lowrank_flops_literal_hand_count():
    # m = n = 10, l = 4, r = 2, q = 1, by hand:
    #   products with A: Y = A Omega, A^T Q, A Q~, A^T Q  -> 4 x 2 x 10 x 10 x 4 = 3200
    #   QRs: 4 panels of 10 x 4, each 2 (2 * 16 * (10 - 4/3)) = 2 x 277.33.. = 554.66..
    #        -> 2218.66.. (exactly 6656/3)
    #   final products U (10 x 4 by 4 x 2) and V (10 x 4 by 4 x 2): 160 + 160 = 320
    #   total 3200 + 6656/3 + 320 = 17216/3
    assert L.lowrank_flops(10, 10, 4, 2, 1) == pytest.approx(17216 / 3, rel=1e-15)
    # m = 1024, n = 1024, l = 26, r = 16, q = 1 (the benchmark's blocks):
    #   4 x 2 x 1024^2 x 26 = 218103808; QRs: 4 panels of 1024 x 26, each
    #   2 x 2 x 676 x (1024 - 26/3), together 10816 x 3046/3 = 32945536/3;
    #   final 2 x 2 x 1024 x 26 x 16 = 1703936
    assert L.lowrank_flops(1024, 1024, 26, 16, 1) == pytest.approx(218103808 + 32945536 / 3 + 1703936, rel=1e-15)
