"""Oracle for the producers and consumers of low-rank blocks.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
benchmark's CPU-baseline leg; never by the library.  Plain numpy in binary64;
numpy's matmul, QR and SVD serve as single steps, nothing is blocked, fused or
reordered beyond the algorithms stated here.

A block of shape (m, n, rank) is stored as A ~= U S V (Eq. 1, Sec. 2): U is
m x r, S is r x r (here diagonal, given by its r values), V is r x n.  Sec. 2
names the producers and consumers around the batched low-rank product:

* randomized SVD (Sec. 2 cites Halko, Martinsson and Tropp, "Finding structure
  with randomness", 2009/2011) produces U, S, V from a dense block:
    - stage A, randomized range finder: Y = A Omega for an n x l Gaussian test
      matrix Omega (l = r + oversampling), Q = orthonormal basis of range(Y);
      with q power (subspace) iterations, alternate Q~ = orth(A^T Q) and
      Q = orth(A Q~) q times, re-orthonormalising after every product;
    - stage B, direct SVD: B = Q^T A (l x n), B = U~ Sigma W^T, U = Q U~;
      keep the r leading singular triplets: U = Q U~[:, :r], S = Sigma[:r],
      V = W^T[:r, :].
  The test matrix is an input (the random numbers the method draws), so the
  oracle and the GPU path see the same Omega.
* expansion back to a dense block: D <- D + U diag(S) V (Eq. 1), computed as
  (U diag(S)) V: the columns of U scaled first, then one product.
* rounded addition (Sec. 2 cites Bebendorf's stabilised rounded addition, whose
  first step is the low-rank product): the sum of two low-rank blocks
  U1 S1 V1 + U2 S2 V2, truncated to rank r, by the standard route:
  Uc = [U1 diag(S1), U2 diag(S2)] = Q1 R1,  Vc^T = [V1; V2]^T = Q2 R2,
  R1 R2^T = U~ Sigma W^T,  U = Q1 U~[:, :r], S = Sigma[:r], V = (Q2 W[:, :r])^T.
"""
from __future__ import annotations

import numpy as np


def orth(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) (m x l, m >= l): the Q of a thin QR."""
    Q, _ = np.linalg.qr(Y, mode="reduced")
    return Q


def range_finder(A: np.ndarray, Omega: np.ndarray, q: int = 0) -> np.ndarray:
    """Stage A: Q (m x l) with range(Q) ~ range(A).  q = 0 is the plain range
    finder, q >= 1 randomized subspace iteration (Halko et al., Alg. 4.1 and
    Alg. 4.4)."""
    A = np.asarray(A, dtype=np.float64)
    Q = orth(A @ Omega)
    for _ in range(q):
        Qt = orth(A.T @ Q)
        Q = orth(A @ Qt)
    return Q


def rsvd(A: np.ndarray, Omega: np.ndarray, r: int, q: int = 0):
    """Randomized SVD of one dense block (stage A, then stage B: Halko et al.,
    Alg. 5.1).  Returns U (m x r), S (r,), V (r x n) with A ~= U diag(S) V and
    S in descending order."""
    A = np.asarray(A, dtype=np.float64)
    l = Omega.shape[1]
    if not (1 <= r <= l <= min(A.shape)):
        raise ValueError("need 1 <= r <= l <= min(m, n)")
    Q = range_finder(A, Omega, q)
    B = Q.T @ A
    Ut, sigma, Wt = np.linalg.svd(B, full_matrices=False)
    return Q @ Ut[:, :r], sigma[:r].copy(), Wt[:r, :].copy()


def lr_expand(U: np.ndarray, S: np.ndarray, V: np.ndarray, D: np.ndarray) -> np.ndarray:
    """D + U diag(S) V (Eq. 1): columns of U scaled by S, then one product."""
    return D + (U * S[None, :]) @ V


def lr_round_add(U1, S1, V1, U2, S2, V2, r: int):
    """Rank-r truncation of U1 diag(S1) V1 + U2 diag(S2) V2 through QR of the
    stacked bases and an SVD of the small core R1 R2^T."""
    Uc = np.hstack([U1 * S1[None, :], U2 * S2[None, :]])
    Vc = np.vstack([V1, V2])
    if not (1 <= r <= Uc.shape[1] <= min(Uc.shape[0], Vc.shape[1])):
        raise ValueError("need 1 <= r <= r1 + r2 <= min(m, n)")
    Q1, R1 = np.linalg.qr(Uc, mode="reduced")
    Q2, R2 = np.linalg.qr(Vc.T, mode="reduced")
    Ut, sigma, Wt = np.linalg.svd(R1 @ R2.T)
    return Q1 @ Ut[:, :r], sigma[:r].copy(), (Q2 @ Wt.T[:, :r]).T.copy()


def lowrank_flops(m: int, n: int, l: int, r: int, q: int = 0) -> float:
    """Multiply-add count x 2 of the randomized SVD's products with A and of
    the tall-skinny QRs (Householder, 2 m l^2 - 2 l^3 / 3 each, plus forming Q
    at the same cost) and the final products, as counted for throughput."""
    gemm_a = 2.0 * m * n * l * (2 + 2 * q)
    qr = lambda rows: 2.0 * (2.0 * rows * l * l - 2.0 * l ** 3 / 3.0)
    qrs = (1 + q) * qr(m) + (1 + q) * qr(n)
    final = 2.0 * m * l * r + 2.0 * n * l * r
    return gemm_a + qrs + final
