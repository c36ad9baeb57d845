"""Helpers for comparing the CUDA path with the oracle (test code only)."""
from __future__ import annotations

import numpy as np
import torch

import oracle

REL_FRO_TOL = 1e-13          # per-entry relative Frobenius error of the FP64 path


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu").numpy().copy()


def oracle_batch(Ah, Bh, C0h, batch, entries=None) -> np.ndarray:
    """Full oracle on host copies of the flat buffers; returns the new C buffer."""
    C = C0h.copy()
    idx = range(len(batch)) if entries is None else entries
    ents = [dict(A=Ah, B=Bh, C=C, offA=int(batch.offA[e]), offB=int(batch.offB[e]), offC=int(batch.offC[e]),
                 m=int(batch.m[e]), n=int(batch.n[e]), k=int(batch.k[e]), lda=int(batch.lda[e]),
                 ldb=int(batch.ldb[e]), ldc=int(batch.ldc[e])) for e in idx]
    oracle.gemm_batch(ents)
    return C


def entry_view(buf: np.ndarray, off: int, rows: int, cols: int, ld: int) -> np.ndarray:
    assert off + (cols - 1) * ld + rows <= len(buf)
    it = buf.itemsize
    return np.lib.stride_tricks.as_strided(buf[off:], shape=(rows, cols), strides=(it, it * ld))


def check_entries(Cg, Cexp, Ah, Bh, C0h, batch, entries=None, tol=REL_FRO_TOL):
    """Per entry: relative Frobenius error <= tol and every element within
    2 gamma_{k+1} (|C0| + |A||B|).  Returns the worst relative error."""
    worst = 0.0
    idx = range(len(batch)) if entries is None else entries
    for e in idx:
        m, n, k = int(batch.m[e]), int(batch.n[e]), int(batch.k[e])
        g = entry_view(Cg, int(batch.offC[e]), m, n, int(batch.ldc[e]))
        x = entry_view(Cexp, int(batch.offC[e]), m, n, int(batch.ldc[e]))
        nrm = np.linalg.norm(x)
        err = np.linalg.norm(g - x)
        rel = err / nrm if nrm > 0 else err
        assert rel <= tol, f"entry {e} ({m}x{n}x{k}): rel Frobenius error {rel:.3e}"
        bound = oracle.absbound(m, n, k, Ah, int(batch.offA[e]), int(batch.lda[e]), Bh, int(batch.offB[e]),
                                int(batch.ldb[e]), C0h, int(batch.offC[e]), int(batch.ldc[e]))
        lim = 2 * oracle.gamma(k + 1) * bound * (1 + 2.0 ** -50)
        bad = np.abs(g - x) > lim
        assert not bad.any(), f"entry {e}: {int(bad.sum())} elements outside the rounding-error bound"
        worst = max(worst, rel)
    return worst


def sample_check(batch, Cg_dev: torch.Tensor, C0_samples, samples, tol=REL_FRO_TOL):
    """Check sampled outputs of a device-resident batch against the oracle's
    element sampler.  samples: (entry, i, j) int arrays; C0_samples: old C."""
    ents, ii, jj = samples
    k_all = batch.k[ents]
    errs, mags = [], []
    for kk in np.unique(k_all):
        sel = np.nonzero(k_all == kk)[0]
        e, i, j = ents[sel], ii[sel], jj[sel]
        p = np.arange(kk)
        a_idx = batch.offA[e][:, None] + i[:, None] + p[None, :] * batch.lda[e][:, None]
        b_idx = batch.offB[e][:, None] + p[None, :] + j[:, None] * batch.ldb[e][:, None]
        arow = batch.A[torch.as_tensor(a_idx.ravel(), device=batch.A.device)].cpu().numpy().reshape(len(sel), kk)
        bcol = batch.B[torch.as_tensor(b_idx.ravel(), device=batch.B.device)].cpu().numpy().reshape(len(sel), kk)
        c0 = C0_samples[sel]
        exp = oracle.gemm_elements(arow, bcol, c0)
        c_idx = batch.offC[e] + i + j * batch.ldc[e]
        got = Cg_dev[torch.as_tensor(c_idx, device=Cg_dev.device)].cpu().numpy()
        bound = np.abs(c0) + np.sum(np.abs(arow) * np.abs(bcol), axis=1)
        lim = 2 * oracle.gamma(int(kk) + 1) * bound * (1 + 2.0 ** -50)
        assert np.all(np.abs(got - exp) <= lim), f"k={kk}: sampled element outside the rounding-error bound"
        errs.append(got - exp)
        mags.append(exp)
    err = np.concatenate(errs)
    mag = np.concatenate(mags)
    rel = np.linalg.norm(err) / np.linalg.norm(mag)
    assert rel <= tol, f"sampled relative error {rel:.3e}"
    return rel


def draw_samples(batch, count, seed=0, extra_entries=()):
    rng = np.random.default_rng(seed)
    ents = rng.integers(0, len(batch), count)
    ents = np.concatenate([ents, np.asarray(extra_entries, dtype=np.int64)])
    ii = (rng.random(len(ents)) * batch.m[ents]).astype(np.int64)
    jj = (rng.random(len(ents)) * batch.n[ents]).astype(np.int64)
    # corners: last row / last column of the sampled entries
    ii[::7] = batch.m[ents[::7]] - 1
    jj[::5] = batch.n[ents[::5]] - 1
    return ents.astype(np.int64), ii, jj


def c0_at(batch, samples):
    ents, ii, jj = samples
    c_idx = batch.offC[ents] + ii + jj * batch.ldc[ents]
    return batch.C[torch.as_tensor(c_idx, device=batch.C.device)].cpu().numpy()
