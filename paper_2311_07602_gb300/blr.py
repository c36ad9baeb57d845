"""Block low-rank (BLR) matrix times several right-hand sides, on the library.

The paper's application benchmark (Sec. 7, BLR matrix-vector product): a
weakly admissible BLR matrix of order N = nb * b has dense diagonal blocks
D_i (b x b) and low-rank off-diagonal blocks A_ij = U_ij S_ij V_ij
(b x r, r x r, r x b; Eq. 1); Y += A X for X with nrhs columns is

    Y_i += D_i X_i + sum_{j != i} U_ij (S_ij (V_ij X_j)).

Three batched calls of the library, nothing else on the path:
  1. the diagonal blocks, a T-form batch (b x b) (b x nrhs);
  2. T_ij = S_ij (V_ij X_j) for every off-diagonal block -- the low-rank
     chain of Alg. 1 with A_X = S_ij, A_{V^T} = V_ij, B_U = X_j, B_X = I --
     written into a per-row stack T_i = [T_ij]_j ((nb-1) r x nrhs);
  3. Y_i += [U_ij]_j T_i, one product per block row with k = (nb-1) r, the
     U blocks of a row stored side by side.
Steps 1 and 2 touch disjoint outputs (Y and the stacks T) and run on two
streams at once; step 3 waits for both.  Step 3 gives every block row one
entry, so no two entries write the same part of Y.  Y's blocks interleave in
memory (ld = N), so the byte-range alias check, which is conservative, is
switched off for steps 1 and 3.

The block rows are split into groups, each with its own three plans, so
that step 3 of one group (a few long-k products that alone would leave a
tail of idle SMs) overlaps step 2 of the next: the chains of all groups run
in order on one stream, and each group has a stream of its own for step 1
and, once that group's chains are done, step 3 (the long-k tiles of step 3
are latency-bound, so the groups' steps 3 must overlap one another too).
Groups write disjoint rows of Y and disjoint stacks T.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import lrbatch as L


@dataclass
class BLRMatrix:
    nb: int
    b: int
    r: int
    D: torch.Tensor       # nb blocks b x b, column-major, back to back
    U: torch.Tensor       # per block row i: b x (nb-1) r panel [U_ij]_{j != i}, column-major, ld b
    S: torch.Tensor       # nb (nb-1) blocks r x r, ordered (i, j != i)
    V: torch.Tensor       # nb (nb-1) blocks r x b, same order

    @property
    def N(self):
        return self.nb * self.b

    def flops(self, nrhs: int) -> float:
        nb, b, r = self.nb, self.b, self.r
        lr = nb * (nb - 1) * (2.0 * r * b * nrhs + 2.0 * r * r * nrhs) + nb * 2.0 * b * (nb - 1) * r * nrhs
        return nb * 2.0 * b * b * nrhs + lr


def random_blr(nb: int, b: int, r: int, seed: int = 0, device="cpu") -> BLRMatrix:
    """N(0,1) dense diagonal blocks and factors (the paper's experiments use
    normally distributed entries), S scaled by 1/sqrt(b) so blocks stay O(1)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = dict(dtype=torch.float64, device=device)
    D = torch.empty(nb * b * b, **f64).normal_(generator=g)
    U = torch.empty(nb * b * (nb - 1) * r, **f64).normal_(generator=g)
    S = torch.empty(nb * (nb - 1) * r * r, **f64).normal_(generator=g).mul_(1.0 / np.sqrt(b))
    V = torch.empty(nb * (nb - 1) * r * b, **f64).normal_(generator=g)
    return BLRMatrix(nb, b, r, D, U, S, V)


class BLRMatVec:
    """Plans of Y += A X for a BLR matrix and fixed X / Y buffers (device,
    column-major N x nrhs with leading dimension N).  fused selects the fused
    low-rank chain kernel (ranks <= 64) or the three-product comparator;
    groups is the number of block-row groups pipelined against each other."""

    def __init__(self, handle: L.Handle, M: BLRMatrix, X: torch.Tensor, Y: torch.Tensor, nrhs: int,
                 fused: bool = True, groups: int = 2):
        nb, b, r, N = M.nb, M.b, M.r, M.N
        self.M, self.nrhs = M, nrhs
        dev = X.device
        self.T = torch.zeros(nb * (nb - 1) * r * nrhs, dtype=torch.float64, device=dev)
        self.I = torch.eye(nrhs, dtype=torch.float64, device=dev).reshape(-1).contiguous()
        x0, y0, t0 = X.data_ptr(), Y.data_ptr(), self.T.data_ptr()
        # 1. diagonal blocks
        d1 = np.zeros(nb, dtype=L.DESC_DTYPE)
        i = np.arange(nb, dtype=np.uint64)
        d1["A"] = np.uint64(M.D.data_ptr()) + 8 * i * np.uint64(b * b)
        d1["B"] = np.uint64(x0) + 8 * i * np.uint64(b)
        d1["C"] = np.uint64(y0) + 8 * i * np.uint64(b)
        d1["m"], d1["n"], d1["k"], d1["lda"], d1["ldb"], d1["ldc"] = b, nrhs, b, b, N, N
        # 2. T_ij = S_ij (V_ij X_j), stacked per block row
        cnt = nb * (nb - 1)
        d2 = np.zeros(cnt, dtype=L.LR_DESC_DTYPE)
        ii = np.repeat(np.arange(nb), nb - 1)
        jpos = np.tile(np.arange(nb - 1), nb)
        jj = jpos + (jpos >= ii)                      # skip the diagonal
        q = np.arange(cnt, dtype=np.uint64)
        d2["AVT"] = np.uint64(M.V.data_ptr()) + 8 * q * np.uint64(r * b)
        d2["BU"] = np.uint64(x0) + 8 * jj.astype(np.uint64) * np.uint64(b)
        d2["AX"] = np.uint64(M.S.data_ptr()) + 8 * q * np.uint64(r * r)
        d2["BX"] = np.uint64(self.I.data_ptr())
        d2["G"] = np.uint64(t0) + 8 * (ii.astype(np.uint64) * np.uint64((nb - 1) * r * nrhs) +
                                       jpos.astype(np.uint64) * np.uint64(r))
        d2["ra"], d2["rb"], d2["k"] = r, nrhs, b
        d2["ld_avt"], d2["ld_bu"], d2["ld_ax"], d2["ld_bx"], d2["ldg"] = r, N, r, nrhs, (nb - 1) * r
        # 3. Y_i += [U_ij]_j T_i
        d3 = np.zeros(nb, dtype=L.DESC_DTYPE)
        d3["A"] = np.uint64(M.U.data_ptr()) + 8 * i * np.uint64(b * (nb - 1) * r)
        d3["B"] = np.uint64(t0) + 8 * i * np.uint64((nb - 1) * r * nrhs)
        d3["C"] = np.uint64(y0) + 8 * i * np.uint64(b)
        d3["m"], d3["n"], d3["k"], d3["lda"], d3["ldb"], d3["ldc"] = b, nrhs, (nb - 1) * r, b, (nb - 1) * r, N
        self.side = None
        self.plans = []
        for rows in np.array_split(np.arange(nb), max(1, min(groups, nb))):
            i0, i1 = int(rows[0]), int(rows[-1]) + 1
            q0, q1 = i0 * (nb - 1), i1 * (nb - 1)
            self.plans.append((handle.plan(d1[i0:i1], check_alias=False, use_graph=True),
                               L.Plan(handle, d2[q0:q1], lr_fused=fused),
                               handle.plan(d3[i0:i1], check_alias=False, use_graph=True)))

    def run(self, stream=None):
        # steps 1 and 2 write different buffers (Y, T), so they run concurrently:
        # the chains fill the SMs the diagonal products leave idle, and a
        # group's step 3 overlaps the next groups' chains and steps 3
        s = stream if stream is not None else torch.cuda.current_stream()
        if self.side is None:
            self.side = torch.cuda.Stream(device=s.device)
            self.rows = [torch.cuda.Stream(device=s.device) for _ in self.plans]
            self.ev_fork = torch.cuda.Event()
            self.ev_chains = [torch.cuda.Event() for _ in self.plans]
            self.ev_rows = [torch.cuda.Event() for _ in self.plans]
        self.ev_fork.record(s)
        self.side.wait_event(self.ev_fork)
        for (_, p2, _), ev in zip(self.plans, self.ev_chains):
            p2.launch(self.side)
            ev.record(self.side)
        for (p1, _, p3), rs, ev, done in zip(self.plans, self.rows, self.ev_chains, self.ev_rows):
            rs.wait_event(self.ev_fork)
            p1.launch(rs)
            rs.wait_event(ev)
            p3.launch(rs)
            done.record(rs)
        for done in self.ev_rows:
            s.wait_event(done)

    def close(self):
        for group in self.plans:
            for p in group:
                p.close()
