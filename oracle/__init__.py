"""The oracle: a plain, slow CPU statement of batched C_i += A_i * B_i.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA
library and does not import it.

* FP64 (oracle_gemm.c, via ctypes): the per-entry triple loop of Alg. 1's
  first step / Alg. 2 loops 1-4, binary64, old C plus products in increasing
  k, no fused multiply-add.
* Split precision (split.py): the Ozaki-style digit splitting, exact int64
  digit products and binary64 recombination.
* Low-rank producers and consumers (lowrank.py): randomized SVD of a dense
  block, expansion U diag(S) V, rounded addition of two low-rank blocks.

Arrays are numpy float64, column-major views described by (m, n, k, ld).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from .split import (PRESETS, SplitParams, apriori_bound, chunk_exponents,  # noqa: F401
                    chunk_level_sums, level_bound, recombination_magnitude,
                    reconstruct, split_digits, split_dot_samples, split_gemm)

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        L.oracle_gemm.argtypes = [i32, i32, i32, _dp, i32, _dp, i32, _dp, i32]
        L.oracle_gemm.restype = None
        L.oracle_gemm_batch.argtypes = [i64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int]
        L.oracle_gemm_batch.restype = ctypes.c_int
        L.oracle_gemm_elements.argtypes = [i64, i32, _dp, _dp, _dp, _dp]
        L.oracle_gemm_elements.restype = None
        L.oracle_gemm_absbound.argtypes = [i32, i32, i32, _dp, i32, _dp, i32, _dp, i32, _dp]
        L.oracle_gemm_absbound.restype = None
        L.oracle_lr_chain.argtypes = [i32, i32, i32, _dp, i32, _dp, i32, _dp, i32, _dp, i32, _dp, i32, _dp]
        L.oracle_lr_chain.restype = None
        L.oracle_lr_chain_batch.argtypes = [i64] + [ctypes.c_void_p] * 8 + [ctypes.c_int]
        L.oracle_lr_chain_batch.restype = ctypes.c_int
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray, offset_elems: int = 0):
    return ctypes.cast(a.ctypes.data + 8 * offset_elems, _dp)


def _check_buf(buf: np.ndarray):
    if buf.dtype != np.float64 or not buf.flags.c_contiguous:
        raise ValueError("oracle buffers must be contiguous float64")


def gemm(m, n, k, A, offA, lda, B, offB, ldb, C, offC, ldc):
    """One entry on flat buffers: C[offC + i + j*ldc] += sum_p A[offA+i+p*lda]*B[offB+p+j*ldb]."""
    for buf in (A, B, C):
        _check_buf(buf)
    lib().oracle_gemm(m, n, k, _ptr(A, offA), lda, _ptr(B, offB), ldb, _ptr(C, offC), ldc)


def gemm_batch(entries, nthreads: int = 0) -> int:
    """entries: list of dicts with keys A, B, C (flat float64 numpy buffers),
    offA, offB, offC (element offsets), m, n, k, lda, ldb, ldc.
    Updates each C in place; returns the OpenMP thread count used."""
    cnt = len(entries)
    if cnt == 0:
        return 0
    pa = (ctypes.c_void_p * cnt)()
    pb = (ctypes.c_void_p * cnt)()
    pc = (ctypes.c_void_p * cnt)()
    dims = {key: np.zeros(cnt, dtype=np.int32) for key in ("m", "n", "k", "lda", "ldb", "ldc")}
    for e, d in enumerate(entries):
        for buf in (d["A"], d["B"], d["C"]):
            _check_buf(buf)
        pa[e] = d["A"].ctypes.data + 8 * d.get("offA", 0)
        pb[e] = d["B"].ctypes.data + 8 * d.get("offB", 0)
        pc[e] = d["C"].ctypes.data + 8 * d.get("offC", 0)
        for key in dims:
            dims[key][e] = d[key]
    return lib().oracle_gemm_batch(cnt, pa, pb, pc, *(dims[key].ctypes.data for key in
                                   ("m", "n", "k", "lda", "ldb", "ldc")), nthreads)


def gemm_elements(arow: np.ndarray, bcol: np.ndarray, c0: np.ndarray) -> np.ndarray:
    """Selected outputs: arow (q, k) rows of A, bcol (q, k) columns of B,
    c0 (q,) old C values -> (q,) new values, same summation as gemm."""
    arow = np.ascontiguousarray(arow, dtype=np.float64)
    bcol = np.ascontiguousarray(bcol, dtype=np.float64)
    c0 = np.ascontiguousarray(c0, dtype=np.float64)
    q, k = arow.shape
    out = np.empty(q, dtype=np.float64)
    lib().oracle_gemm_elements(q, k, _ptr(arow), _ptr(bcol), _ptr(c0), _ptr(out))
    return out


def absbound(m, n, k, A, offA, lda, B, offB, ldb, C0, offC, ldc) -> np.ndarray:
    """|C0| + |A| |B| as an (m, n) column-major array (binary64, unrounded-up)."""
    out = np.empty(m * n, dtype=np.float64)
    lib().oracle_gemm_absbound(m, n, k, _ptr(A, offA), lda, _ptr(B, offB), ldb,
                               _ptr(C0, offC), ldc, _ptr(out))
    return out.reshape(n, m).T


def lr_chain(AVT: np.ndarray, BU: np.ndarray, AX: np.ndarray, BX: np.ndarray) -> np.ndarray:
    """G = A_X (A_{V^T} B_U) B_X for one entry (Alg. 1); 2-D float64 arrays,
    any memory order; returns G (ra x rb)."""
    ra, k = AVT.shape
    rb = BU.shape[1]
    f = lambda x: np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel(order="F"))
    a, b, x, y = f(AVT), f(BU), f(AX), f(BX)
    G = np.zeros(ra * rb)
    work = np.zeros(2 * ra * rb)
    lib().oracle_lr_chain(ra, rb, k, _ptr(a), ra, _ptr(b), k, _ptr(x), ra, _ptr(y), rb, _ptr(G), ra, _ptr(work))
    return G.reshape(rb, ra).T


def lr_chain_batch(bufs: dict, offs: dict, ra, rb, k, nthreads: int = 0) -> int:
    """Chains on flat buffers: bufs/offs keyed AVT, BU, AX, BX, G (tight
    leading dimensions); per-entry arrays ra, rb, k.  Writes G in place."""
    cnt = len(ra)
    arrs = {}
    for key in ("AVT", "BU", "AX", "BX", "G"):
        _check_buf(bufs[key])
        p = (ctypes.c_void_p * cnt)()
        base = bufs[key].ctypes.data
        for e in range(cnt):
            p[e] = base + 8 * int(offs[key][e])
        arrs[key] = p
    dims = [np.ascontiguousarray(x, dtype=np.int32) for x in (ra, rb, k)]
    return lib().oracle_lr_chain_batch(cnt, arrs["AVT"], arrs["BU"], arrs["AX"], arrs["BX"], arrs["G"],
                                       *(d.ctypes.data for d in dims), nthreads)


def max_threads() -> int:
    return lib().oracle_max_threads()


def gamma(n: int) -> float:
    """Higham's gamma_n = n u / (1 - n u), u = 2^-53 (unit roundoff of binary64)."""
    u = 2.0 ** -53
    return n * u / (1.0 - n * u)
