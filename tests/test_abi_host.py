"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every function include/lrbatch.h declares; argument validation
returns status codes before any CUDA call; the planner's tile list covers
every output element of every entry exactly once."""
import ctypes

import numpy as np
import pytest

from paper_2311_07602_gb300 import lrbatch as L


def test_exports_every_declared_symbol():
    lib = L.lib()
    declared = L.declared_functions()
    assert "lrb_plan_create" in declared and "lrb_launch" in declared
    for name in declared:
        assert hasattr(lib, name), name


def descs(*rows):
    d = np.zeros(len(rows), dtype=L.DESC_DTYPE)
    for i, r in enumerate(rows):
        d[i] = r
    return d


GOOD = (0x100000, 0x200000, 0x300000, 4, 3, 2, 4, 2, 4)


@pytest.mark.parametrize("bad,status", [
    ((0, 0x200000, 0x300000, 4, 3, 2, 4, 2, 4), L.LRB_ERR_INVALID),        # NULL A
    ((0x100000, 0x200000, 0, 4, 3, 2, 4, 2, 4), L.LRB_ERR_INVALID),        # NULL C
    ((0x100000, 0x200000, 0x300000, 0, 3, 2, 4, 2, 4), L.LRB_ERR_INVALID),  # m = 0
    ((0x100000, 0x200000, 0x300000, 4, -1, 2, 4, 2, 4), L.LRB_ERR_INVALID),  # n < 0
    ((0x100000, 0x200000, 0x300000, 4, 3, 2, 3, 2, 4), L.LRB_ERR_INVALID),  # lda < m
    ((0x100000, 0x200000, 0x300000, 4, 3, 2, 4, 1, 4), L.LRB_ERR_INVALID),  # ldb < k
    ((0x100000, 0x200000, 0x300000, 4, 3, 2, 4, 2, 3), L.LRB_ERR_INVALID),  # ldc < m
    ((0x100004, 0x200000, 0x300000, 4, 3, 2, 4, 2, 4), L.LRB_ERR_INVALID),  # misaligned A
    ((0xFFFFFFFFFFFF0000, 0x200000, 0x300000, 4, 3, 2**30, 4, 2**30, 4), L.LRB_ERR_INVALID),  # wraps
])
def test_validation_status_codes(bad, status):
    assert L.lrb_validate(descs(GOOD)) == L.LRB_OK
    assert L.lrb_validate(descs(GOOD, bad)) == status
    assert L.last_error() != ""


def test_validation_count_and_null():
    assert L.lib().lrb_validate(None, 1, None) == L.LRB_ERR_INVALID
    d = descs(GOOD)
    assert L.lib().lrb_validate(d.ctypes.data, 0, None) == L.LRB_ERR_INVALID
    o = L.make_opts(precision=99)
    assert L.lrb_validate(d, o) == L.LRB_ERR_INVALID
    o = L.make_opts(force_variant=L.lrb_variant_count())
    assert L.lrb_validate(d, o) == L.LRB_ERR_INVALID


def test_alias_detection():
    # C of entry 1 overlaps C of entry 0 (4x3, ldc 4 -> 96 bytes)
    a = (0x100000, 0x200000, 0x300000, 4, 3, 2, 4, 2, 4)
    b = (0x100000, 0x200000, 0x300000 + 88, 4, 3, 2, 4, 2, 4)
    assert L.lrb_validate(descs(a, b)) == L.LRB_ERR_ALIAS
    c = (0x100000, 0x200000, 0x300000 + 96, 4, 3, 2, 4, 2, 4)       # adjacent: fine
    assert L.lrb_validate(descs(a, c)) == L.LRB_OK
    # an operand of one entry overlaps another entry's C
    d = (0x300000 + 40, 0x200000, 0x500000, 4, 3, 2, 4, 2, 4)
    assert L.lrb_validate(descs(a, d)) == L.LRB_ERR_ALIAS
    # shared A/B between entries is allowed
    e = (0x100000, 0x200000, 0x600000, 4, 3, 2, 4, 2, 4)
    assert L.lrb_validate(descs(a, e)) == L.LRB_OK
    # alias check can be switched off
    assert L.lrb_validate(descs(a, b), L.make_opts(check_alias=False)) == L.LRB_OK


@pytest.mark.parametrize("variant", range(10))
def test_tiles_cover_every_output_once(variant):
    rng = np.random.default_rng(variant)
    shapes = [(int(rng.integers(1, 300)), int(rng.integers(1, 200)), int(rng.integers(1, 50))) for _ in range(40)]
    shapes += [(1, 1, 1), (64, 64, 16), (2048, 128, 2048)]
    rows = []
    base = 0x10000000
    for i, (m, n, k) in enumerate(shapes):
        rows.append((base, base, base + (i + 1) * 0x4000000, m, n, k, m, k, m))
    d = descs(*rows)
    tiles = L.lrb_plan_tiles_host(d, variant)
    bm, bn, _ = L.lrb_variant_shape(variant)
    cover = [np.zeros((m, n), dtype=np.int32) for m, n, k in shapes]
    for e, r0, c0, h, w in tiles:
        assert 0 < h <= bm and 0 < w <= bn
        cover[e][r0:r0 + h, c0:c0 + w] += 1
    for c in cover:
        assert np.all(c == 1)
    # longest-first: tile costs never increase along the list
    k = np.array([shapes[e][2] for e in tiles[:, 0]], dtype=np.float64)
    hh = tiles[:, 3].astype(np.float64)
    if _ := L.lrb_variant_shape(variant)[2]:
        cost = np.ceil(hh / 8) * 8 * np.ceil(tiles[:, 4] / 8) * 8 * np.ceil(k / 4) * 4
    else:
        cost = np.ceil(hh / 32) * 32 * tiles[:, 4] * k
    assert np.all(np.diff(cost) <= 0)


def test_transposed_forms_validate_stored_shapes():
    # m = 4, n = 3, k = 2.  A^T: A stored k x m (lda >= k = 2); B^T: B stored n x k (ldb >= n = 3)
    base = (0x100000, 0x200000, 0x300000, 4, 3, 2)
    ok = {0: (4, 2, 4), 1: (2, 2, 4), 2: (4, 3, 4), 3: (2, 3, 4)}
    for trans, lds in ok.items():
        o = L.make_opts(trans=trans)
        assert L.lrb_validate(descs(base + lds), o) == L.LRB_OK, trans
    # lda = 2 < m is fine only when A is transposed; ldb = 2 < n fails when B is
    assert L.lrb_validate(descs(base + (2, 2, 4)), L.make_opts(trans=0)) == L.LRB_ERR_INVALID
    assert L.lrb_validate(descs(base + (4, 2, 4)), L.make_opts(trans=2)) == L.LRB_ERR_INVALID
    assert L.lrb_validate(descs(base + (1, 3, 4)), L.make_opts(trans=3)) == L.LRB_ERR_INVALID
    assert L.lrb_validate(descs(base + (4, 2, 4)), L.make_opts(trans=4)) == L.LRB_ERR_INVALID
    o = L.make_opts()
    o.overwrite = 2
    assert L.lrb_validate(descs(base + (4, 2, 4)), o) == L.LRB_ERR_INVALID


def test_transposed_alias_uses_stored_extent():
    # m = 2, n = 1, k = 3, lda = 10.  A as stored m x k spans 10*(3-1)+2 = 22
    # elements; A^T stored k x m spans 10*(2-1)+3 = 13.  A C at element 15
    # overlaps only the first.
    A = 0x100000
    d = descs((A, 0x200000, A + 8 * 15, 2, 1, 3, 10, 3, 2))
    assert L.lrb_validate(d, L.make_opts(trans=0)) == L.LRB_ERR_ALIAS
    assert L.lrb_validate(d, L.make_opts(trans=1)) == L.LRB_OK
