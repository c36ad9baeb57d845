"""The metric accounting follows the paper's formulas (tests/golden/
paper_accounting.json, written from the Sec. 7 equations): the low-rank
chain workload's flop count equals batch (4 r^3 + 2 r^2 b) and the chain's
executed flops reduce to it for ra = rb = r; the GEMM flop / byte counts of
the workload module are 2 m n k and 8 (mk + kn + 2mn)."""
import json
import os

import numpy as np

from paper_2311_07602_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_accounting.json")


def test_lr_flops_match_paper_formula():
    cases = json.load(open(GOLDEN))["cases"]
    assert len(cases) >= 6
    for c in cases:
        r, b, batch = c["r"], c["b"], c["batch"]
        lb = W.LrBatch({}, {}, np.full(batch, r, np.int32), np.full(batch, r, np.int32), np.full(batch, b, np.int32))
        assert lb.flops_paper() == c["flops"]
        # the chain as executed (ra rb (2k + 2ra + 2rb)) is the paper's count for ra = rb = r
        assert batch * r * r * (2 * b + 4 * r) == c["flops"]
        assert c["bytes_2r2"] == batch * (2 * r * r + 2 * r * b) * 8
        assert c["bytes_3r2"] - c["bytes_2r2"] == batch * r * r * 8


def test_gemm_accounting():
    b = W.uniform_batch(W.FORM_T, 64, 8, 3, seed=1)
    assert b.flops() == 3 * 2 * 64 * 8 * 64
    assert b.alg_bytes() == 3 * 8 * (64 * 64 + 64 * 8 + 2 * 64 * 8)
    o = W.small_o_form()
    assert o.flops() == 64 * 2 * 256 * 256 * 16 == 134217728
    assert o.alg_bytes() == 64 * 8 * (256 * 16 + 16 * 256 + 2 * 256 * 256) == 71303168
