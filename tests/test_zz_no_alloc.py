"""lrb_launch_noalloc: the batch without any device allocation.

Some callers cannot call cudaMalloc: their GPU memory is owned by a
framework's pool or a fixed budget set at start-up, or their loop must not
risk the device-wide synchronisation an allocation can cause.  This entry
point keeps its scratch (descriptor copy, tile list, work counter) in a
fixed array inside the library.

The GPU test runs it twice in a row, through the C ABI, on fresh copies of
one mixed batch and checks each result bitwise against the planned launch
with untuned tiles (lrb_plan_create with tune = 0 + lrb_launch: the same tile
rule, so the same tiles and the same summation order) and against the FP64
oracle within the tolerance of the other FP64 tests.  The refusal of
oversize batches is checked without a GPU: it happens before any CUDA call.
The file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2311_07602_gb300 import lrbatch as L
from paper_2311_07602_gb300 import workloads as W
from tests.parity import check_entries, host, oracle_batch


@pytest.mark.gpu
def test_noalloc_matches_planned_launch_and_oracle_on_two_calls():
    forms, bs, rs = W.variable_shapes(300, seed=77, bmin=16, bmax=700)
    base = W.variable_batch(forms, bs, rs, seed=77)
    Ah, Bh, C0 = host(base.A), host(base.B), host(base.C)
    ref_dev = base.to("cuda")
    with L.Handle(0) as h:
        with h.plan(L.descs_for(ref_dev), tune=False) as p:
            # enough tiles that the planner keeps its 64-row untuned tiles
            # (it halves them only below two waves of the persistent grid)
            assert p.info()["items"] >= 2 * 5 * torch.cuda.get_device_properties(0).multi_processor_count
            p.launch()
            torch.cuda.synchronize()
    ref = host(ref_dev.C)
    exp = oracle_batch(Ah, Bh, C0, base)
    for call in range(2):
        dev = base.to("cuda")
        status = L.lrb_launch_noalloc(L.descs_for(dev))
        assert status == L.LRB_OK, L.last_error()
        torch.cuda.synchronize()
        got = host(dev.C)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), f"call {call}: differs from the planned launch"
        check_entries(got, exp, Ah, Bh, C0, base)


def test_noalloc_rejects_oversize_batches():
    d = np.zeros(L.NOALLOC_MAX_ENTRIES + 1, dtype=L.DESC_DTYPE)
    d["A"], d["B"], d["C"] = 0x1000, 0x2000, 0x3000
    d["m"] = d["n"] = d["k"] = d["lda"] = d["ldb"] = d["ldc"] = 1
    assert L.lrb_launch_noalloc(d, stream=0) == L.LRB_ERR_INVALID
    assert "maximum" in L.last_error()
    # within the entry limit but beyond the tile limit, with output widths in
    # every bucket of the tile rule (n <= 8, 16, 32 and wider): the rule the
    # call checks against the planner's must agree for all four variants
    # before the tile count refuses the batch
    d = d[:L.NOALLOC_MAX_ENTRIES].copy()
    d["C"] = 0x10000000 + np.arange(len(d), dtype=np.uint64) * np.uint64(2048 * 1024 * 8)
    d["m"] = d["lda"] = d["ldc"] = 2048
    d["n"] = np.array([5, 16, 30, 1024], dtype=np.int32)[np.arange(len(d)) % 4]
    assert L.lrb_launch_noalloc(d, stream=0) == L.LRB_ERR_INVALID
    assert "tiles" in L.last_error()
