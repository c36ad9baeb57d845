"""Pins for the low-rank chain oracle (oracle_lr_chain, Alg. 1:
G = A_X (A_{V^T} B_U) B_X), each against something other than itself:

* identity factors reduce the chain to its first product; permutation
  factors permute rows/columns of it -- exactly, for integer data;
* integer-valued inputs: the exact integer chain (numpy int64);
* the other association (A_X A_{V^T}) (B_U B_X) through numpy, within the
  rounding bounds of both evaluation orders;
* exact rational arithmetic on tiny random inputs, within Higham's bound
  for three chained products;
* the batch entry point equals the single-entry one.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def ints(rng, shape, lo=-8, hi=9):
    return rng.integers(lo, hi, shape).astype(np.float64)


@pytest.mark.parametrize("ra,rb,k", [(1, 1, 1), (4, 3, 9), (8, 8, 64), (16, 32, 100)])
def test_identity_and_permutation_factors(ra, rb, k):
    rng = np.random.default_rng(ra * 100 + rb)
    AVT, BU = ints(rng, (ra, k)), ints(rng, (k, rb))
    first = AVT.astype(np.int64) @ BU.astype(np.int64)
    assert np.array_equal(oracle.lr_chain(AVT, BU, np.eye(ra), np.eye(rb)), first.astype(np.float64))
    P = np.eye(ra)[rng.permutation(ra)]
    Q = np.eye(rb)[rng.permutation(rb)]
    assert np.array_equal(oracle.lr_chain(AVT, BU, P, Q), (P @ first @ Q))


@pytest.mark.parametrize("ra,rb,k", [(8, 8, 512), (16, 16, 128), (5, 7, 33)])
def test_integer_chain_exact(ra, rb, k):
    rng = np.random.default_rng(k)
    AVT, BU, AX, BX = ints(rng, (ra, k), -4, 5), ints(rng, (k, rb), -4, 5), ints(rng, (ra, ra), -3, 4), ints(rng, (rb, rb), -3, 4)
    exact = AX.astype(np.int64) @ (AVT.astype(np.int64) @ BU.astype(np.int64)) @ BX.astype(np.int64)
    assert np.abs(exact).max() < 2 ** 53
    assert np.array_equal(oracle.lr_chain(AVT, BU, AX, BX), exact.astype(np.float64))


def test_other_association_within_bounds():
    rng = np.random.default_rng(3)
    for ra, rb, k in [(8, 8, 512), (32, 32, 1024), (16, 8, 2048)]:
        AVT, BU = rng.standard_normal((ra, k)), rng.standard_normal((k, rb))
        AX, BX = rng.standard_normal((ra, ra)), rng.standard_normal((rb, rb))
        got = oracle.lr_chain(AVT, BU, AX, BX)
        other = (AX @ AVT) @ (BU @ BX)
        mag = np.abs(AX) @ np.abs(AVT) @ np.abs(BU) @ np.abs(BX)
        g = oracle.gamma(k + ra + rb + 3)
        assert np.all(np.abs(got - other) <= 2 * g * mag * (1 + 1e-12))


def test_exact_rational_tiny():
    rng = np.random.default_rng(4)
    u = 2.0 ** -53
    for ra, rb, k in [(1, 1, 1), (2, 3, 4), (3, 2, 5)]:
        AVT, BU = rng.standard_normal((ra, k)), rng.standard_normal((k, rb))
        AX, BX = rng.standard_normal((ra, ra)), rng.standard_normal((rb, rb))
        got = oracle.lr_chain(AVT, BU, AX, BX)
        F = lambda M: [[Fraction(x) for x in row] for row in M]
        def mm(X, Y):
            return [[sum(X[i][p] * Y[p][j] for p in range(len(Y))) for j in range(len(Y[0]))] for i in range(len(X))]
        exact = mm(mm(F(AX), mm(F(AVT), F(BU))), F(BX))
        mag = np.abs(AX) @ np.abs(AVT) @ np.abs(BU) @ np.abs(BX)
        g = oracle.gamma(k + ra + rb)
        for i in range(ra):
            for j in range(rb):
                assert abs(Fraction(got[i, j]) - exact[i][j]) <= Fraction(g * mag[i, j] * (1 + 4 * u))


def test_batch_equals_single():
    rng = np.random.default_rng(5)
    shapes = [(8, 8, 64), (4, 6, 30), (16, 16, 128)]
    bufs = {key: [] for key in ("AVT", "BU", "AX", "BX", "G")}
    offs = {key: [] for key in bufs}
    cur = {key: 0 for key in bufs}
    mats = []
    for ra, rb, k in shapes:
        m = dict(AVT=rng.standard_normal((ra, k)), BU=rng.standard_normal((k, rb)), AX=rng.standard_normal((ra, ra)),
                 BX=rng.standard_normal((rb, rb)), G=np.zeros((ra, rb)))
        mats.append(m)
        for key, X in m.items():
            offs[key].append(cur[key])
            bufs[key].append(X.ravel(order="F"))
            cur[key] += X.size
    flat = {key: np.concatenate(v) for key, v in bufs.items()}
    ra, rb, k = (np.array([s[i] for s in shapes]) for i in range(3))
    assert oracle.lr_chain_batch(flat, offs, ra, rb, k) >= 1
    for e, m in enumerate(mats):
        G = flat["G"][offs["G"][e]:offs["G"][e] + ra[e] * rb[e]].reshape(rb[e], ra[e]).T
        assert np.array_equal(G, oracle.lr_chain(m["AVT"], m["BU"], m["AX"], m["BX"]))
