"""lrb_launch_noalloc: the batch without any device allocation.

Some callers cannot call cudaMalloc: their GPU memory is owned by a
framework's pool or a fixed budget set at start-up, or their loop must not
risk the device-wide synchronisation an allocation can cause.  This entry
point keeps its scratch (descriptor copy, tile list, work counter) in a
fixed array inside the library.  The test runs it twice in a row, through
the C ABI, on fresh copies of one mixed batch and checks each result
against the planned launch (lrb_plan_create + lrb_launch) within the FP64
tolerance used by the other tests; it also checks that oversize batches are
refused with LRB_ERR_INVALID.  The file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2311_07602_gb300 import lrbatch as L
from paper_2311_07602_gb300 import workloads as W
from tests.parity import REL_FRO_TOL, entry_view, host

pytestmark = pytest.mark.gpu


def rel_errors(got, ref, batch):
    out = []
    for e in range(len(batch)):
        m, n, o, ld = int(batch.m[e]), int(batch.n[e]), int(batch.offC[e]), int(batch.ldc[e])
        g = entry_view(got, o, m, n, ld)
        r = entry_view(ref, o, m, n, ld)
        out.append(np.linalg.norm(g - r) / np.linalg.norm(r))
    return np.asarray(out)


def test_noalloc_matches_planned_launch_on_two_calls():
    forms, bs, rs = W.variable_shapes(300, seed=77, bmin=16, bmax=700)
    base = W.variable_batch(forms, bs, rs, seed=77)
    ref_dev = base.to("cuda")
    with L.Handle(0) as h:
        with h.plan(L.descs_for(ref_dev), tune=False) as p:
            p.launch()
            torch.cuda.synchronize()
    ref = host(ref_dev.C)
    for call in range(2):
        dev = base.to("cuda")
        status = L.lrb_launch_noalloc(L.descs_for(dev))
        assert status == L.LRB_OK, L.last_error()
        torch.cuda.synchronize()
        got = host(dev.C)
        errs = rel_errors(got, ref, base)
        assert errs.max() <= REL_FRO_TOL, f"call {call}: max relative error {errs.max():.3e}"


def test_noalloc_rejects_oversize_batches():
    d = np.zeros(L.NOALLOC_MAX_ENTRIES + 1, dtype=L.DESC_DTYPE)
    d["A"], d["B"], d["C"] = 0x1000, 0x2000, 0x3000
    d["m"] = d["n"] = d["k"] = d["lda"] = d["ldb"] = d["ldc"] = 1
    assert L.lrb_launch_noalloc(d) == L.LRB_ERR_INVALID
    assert "maximum" in L.last_error()
    # within the entry limit but beyond the tile limit: 4096 entries of 1024 x 1024 outputs
    d = d[:L.NOALLOC_MAX_ENTRIES].copy()
    d["C"] = 0x10000000 + np.arange(len(d), dtype=np.uint64) * np.uint64(1024 * 1024 * 8)
    d["m"] = d["n"] = d["lda"] = d["ldc"] = 1024
    assert L.lrb_launch_noalloc(d) == L.LRB_ERR_INVALID
    assert "tiles" in L.last_error()
