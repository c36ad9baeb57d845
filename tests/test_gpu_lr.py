"""GPU parity of the batched low-rank chain G = A_X (A_{V^T} B_U) B_X
(Alg. 1) against the oracle, fused (one CTA per block) and unfused (three
batched products), through the C ABI.  Tolerance: relative Frobenius error
<= 1e-13 per block and every element within 2 gamma_{k+ra+rb+2} of
|A_X| |A_{V^T}| |B_U| |B_X|; integer-valued inputs bitwise."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_07602_gb300 import lrbatch as L
from paper_2311_07602_gb300 import workloads as W
from tests.parity import entry_view

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    h = L.Handle(0)
    yield h
    h.close()


def mats(lb, e, host):
    ra, rb, k, pad = int(lb.ra[e]), int(lb.rb[e]), int(lb.k[e]), lb.pad
    v = lambda key, rows, cols: entry_view(host[key], int(lb.offs[key][e]), rows, cols, rows + pad)
    return v("AVT", ra, k), v("BU", k, rb), v("AX", ra, ra), v("BX", rb, rb), v("G", ra, rb)


def run(handle, lb, fused):
    dev = lb.to("cuda")
    with L.Plan(handle, L.lr_descs_for(dev), lr_fused=fused) as p:
        p.launch()
        torch.cuda.synchronize()
    return {key: t.cpu().numpy() for key, t in dev.bufs.items()}


# (ranks chosen so the 2x2 micro-tile count P covers P < 64 with a k-split,
#  64 < P < 128 with idle threads, P = 128 and P > 128 with several per thread)
CASES = [(7, 8, 8, 512), (5, 16, 16, 300), (4, 32, 32, 1024), (3, 9, 13, 77), (2, 64, 64, 256), (2, 1, 1, 1),
         (2, 3, 64, 129), (3, 18, 18, 200), (2, 20, 24, 64), (2, 16, 32, 96), (2, 40, 33, 70)]


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("batch,ra,rb,k", CASES)
def test_chain_matches_oracle(handle, fused, batch, ra, rb, k):
    lb = W.lr_batch(batch, k, ra, rb=rb, seed=ra * 1000 + k, pad=2)
    host = {key: t.numpy().copy() for key, t in lb.bufs.items()}
    G0 = host["G"].copy()
    out = run(handle, lb, fused)
    for e in range(batch):
        AVT, BU, AX, BX, _ = mats(lb, e, host)
        exp = oracle.lr_chain(AVT, BU, AX, BX)
        got = entry_view(out["G"], int(lb.offs["G"][e]), ra, rb, ra + lb.pad)
        rel = np.linalg.norm(got - exp) / np.linalg.norm(exp)
        assert rel <= 1e-13, f"entry {e}: {rel:.3e}"
        mag = np.abs(AX) @ np.abs(AVT) @ np.abs(BU) @ np.abs(BX)
        assert np.all(np.abs(got - exp) <= 2 * oracle.gamma(k + ra + rb + 2) * mag * (1 + 1e-12))
    # only G (not its padding) was written
    written = np.zeros(len(G0), dtype=bool)
    for e in range(batch):
        entry_view(written, int(lb.offs["G"][e]), ra, rb, ra + lb.pad)[...] = True
    assert np.array_equal(out["G"][~written], G0[~written])


@pytest.mark.parametrize("fused", [True, False])
def test_chain_integer_exact(handle, fused):
    lb = W.lr_batch(6, 200, 16, rb=8, seed=9, dist="int8")
    host = {key: t.numpy().copy() for key, t in lb.bufs.items()}
    out = run(handle, lb, fused)
    for e in range(len(lb)):
        AVT, BU, AX, BX, _ = mats(lb, e, host)
        exact = AX.astype(np.int64) @ (AVT.astype(np.int64) @ BU.astype(np.int64)) @ BX.astype(np.int64)
        got = entry_view(out["G"], int(lb.offs["G"][e]), 16, 8, 16)
        assert np.array_equal(got, exact.astype(np.float64))


def test_fused_rank_limit_and_validation(handle):
    lb = W.lr_batch(1, 64, 65, seed=1, device="cuda")
    with pytest.raises(L.LrbError) as ei:
        L.Plan(handle, L.lr_descs_for(lb), lr_fused=True)
    assert ei.value.status == L.LRB_ERR_UNSUPPORTED
    d = L.lr_descs_for(lb)
    d["ldg"] = 3
    with pytest.raises(L.LrbError) as ei:
        L.Plan(handle, d, lr_fused=False)
    assert ei.value.status == L.LRB_ERR_INVALID
