"""Thin ctypes binding of liblrbatch.so (include/lrbatch.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names (lrb_create, lrb_plan_create, ...);
Handle and Plan wrap them for convenience.  Device memory and streams come
from PyTorch (tensor.data_ptr(), stream.cuda_stream).  Loading fails loudly
if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblrbatch.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lrbatch.h")

LRB_OK, LRB_ERR_INVALID, LRB_ERR_ALIAS, LRB_ERR_NOMEM, LRB_ERR_BUDGET, LRB_ERR_QUEUE_FULL, \
    LRB_ERR_TIMEOUT, LRB_ERR_DEVICE, LRB_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = {0: "LRB_OK", 1: "LRB_ERR_INVALID", 2: "LRB_ERR_ALIAS", 3: "LRB_ERR_NOMEM", 4: "LRB_ERR_BUDGET",
                5: "LRB_ERR_QUEUE_FULL", 6: "LRB_ERR_TIMEOUT", 7: "LRB_ERR_DEVICE", 8: "LRB_ERR_UNSUPPORTED"}

LRB_PREC_FP64, LRB_PREC_FP64_DMMA_ALLOWED, LRB_PREC_SPLIT_BF16_S3, LRB_PREC_SPLIT_BF16_S4, \
    LRB_PREC_SPLIT_FP16_S3, LRB_PREC_SPLIT_FP16_S4 = range(6)
SPLIT_PRECISIONS = {"bf16_s3": LRB_PREC_SPLIT_BF16_S3, "bf16_s4": LRB_PREC_SPLIT_BF16_S4,
                    "fp16_s3": LRB_PREC_SPLIT_FP16_S3, "fp16_s4": LRB_PREC_SPLIT_FP16_S4}

# lrb_lr_desc: five pointers then eight int32 (72 bytes)
LR_DESC_DTYPE = np.dtype([("AVT", np.uint64), ("BU", np.uint64), ("AX", np.uint64), ("BX", np.uint64),
                          ("G", np.uint64), ("ra", np.int32), ("rb", np.int32), ("k", np.int32),
                          ("ld_avt", np.int32), ("ld_bu", np.int32), ("ld_ax", np.int32), ("ld_bx", np.int32),
                          ("ldg", np.int32)])
assert LR_DESC_DTYPE.itemsize == 72

# lrb_gemm_desc: three pointers then six int32 (48 bytes, no padding)
DESC_DTYPE = np.dtype([("A", np.uint64), ("B", np.uint64), ("C", np.uint64), ("m", np.int32), ("n", np.int32),
                       ("k", np.int32), ("lda", np.int32), ("ldb", np.int32), ("ldc", np.int32)])
assert DESC_DTYPE.itemsize == 48

# lrb_lr_block: U, S, V pointers then m, n, r, ldu, ldv, reserved (48 bytes)
LR_BLOCK_DTYPE = np.dtype([("U", np.uint64), ("S", np.uint64), ("V", np.uint64), ("m", np.int32), ("n", np.int32),
                           ("r", np.int32), ("ldu", np.int32), ("ldv", np.int32), ("reserved", np.int32)])
assert LR_BLOCK_DTYPE.itemsize == 48
# lrb_rsvd_desc (80 bytes), lrb_expand_desc (64), lrb_round_add_desc (144)
RSVD_DESC_DTYPE = np.dtype([("A", np.uint64), ("Omega", np.uint64), ("out", LR_BLOCK_DTYPE), ("l", np.int32),
                            ("lda", np.int32), ("ldo", np.int32), ("reserved", np.int32)])
assert RSVD_DESC_DTYPE.itemsize == 80
EXPAND_DESC_DTYPE = np.dtype([("blk", LR_BLOCK_DTYPE), ("D", np.uint64), ("ldd", np.int32), ("reserved", np.int32)])
assert EXPAND_DESC_DTYPE.itemsize == 64
ROUND_ADD_DESC_DTYPE = np.dtype([("x", LR_BLOCK_DTYPE), ("y", LR_BLOCK_DTYPE), ("out", LR_BLOCK_DTYPE)])
assert ROUND_ADD_DESC_DTYPE.itemsize == 144
LR_MAX_L = 96          # LRB_LR_MAX_L
LR_MAX_ROWS = 8192     # LRB_LR_MAX_ROWS


class lrb_plan_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("tune", ctypes.c_int32),
                ("force_variant", ctypes.c_int32), ("check_alias", ctypes.c_int32),
                ("test_stall", ctypes.c_int32), ("trans", ctypes.c_int32), ("overwrite", ctypes.c_int32)]


class lrb_plan_info(ctypes.Structure):
    _fields_ = [("entries", ctypes.c_int64), ("items", ctypes.c_int64), ("groups", ctypes.c_int64),
                ("flops", ctypes.c_double), ("alg_bytes", ctypes.c_double), ("grid", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("dmma_items", ctypes.c_int64)]


class lrb_queue_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("accepted", "rejected_budget", "rejected_full", "rejected_invalid",
                                               "completed", "failed", "waiting", "waves", "max_concurrent_waves")] + \
               [("mean_wave_entries", ctypes.c_double)] + \
               [(n, ctypes.c_uint64) for n in ("reserved_bytes", "peak_reserved_bytes", "budget_bytes")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "gflops", "flops_done")]


class lrb_host_timing(ctypes.Structure):
    _fields_ = [("valid", ctypes.c_int32), ("pieces", ctypes.c_int32)] + \
               [(n, ctypes.c_double) for n in ("wall_ms", "h2d_busy_ms", "compute_busy_ms", "d2h_busy_ms",
                                               "h2d_bytes", "d2h_bytes", "overlap_h2d_compute_ms",
                                               "overlap_d2h_compute_ms", "overlap_h2d_d2h_ms", "compute_start_ms",
                                               "compute_end_to_last_ms", "first_h2d_ms", "first_h2d_bytes")]


class LrbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32
        sigs = {
            "lrb_create": ([ctypes.POINTER(vp), ctypes.c_int], i32),
            "lrb_destroy": ([vp], i32),
            "lrb_plan_create": ([vp, vp, sz, ctypes.POINTER(lrb_plan_opts), ctypes.POINTER(vp)], i32),
            "lrb_launch": ([vp, vp], i32),
            "lrb_launch_plain": ([vp, vp], i32),
            "lrb_plan_get_info": ([vp, ctypes.POINTER(lrb_plan_info)], i32),
            "lrb_plan_destroy": ([vp], i32),
            "lrb_validate": ([vp, sz, ctypes.POINTER(lrb_plan_opts)], i32),
            "lrb_execute_host": ([vp, vp, sz, ctypes.POINTER(lrb_plan_opts), vp], i32),
            "lrb_launch_noalloc": ([vp, sz, vp], i32),
            "lrb_plan_status": ([vp], i32),
            "lrb_lr_plan_create": ([vp, vp, sz, i32, ctypes.POINTER(vp)], i32),
            "lrb_rsvd_plan_create": ([vp, vp, sz, i32, ctypes.POINTER(vp)], i32),
            "lrb_expand_plan_create": ([vp, vp, sz, ctypes.POINTER(vp)], i32),
            "lrb_round_add_plan_create": ([vp, vp, sz, ctypes.POINTER(vp)], i32),
            "lrb_queue_create": ([vp, sz, ctypes.c_int, ctypes.POINTER(vp)], i32),
            "lrb_queue_set_limits": ([vp, sz, sz], i32),
            "lrb_queue_set_precision": ([vp, i32], i32),
            "lrb_queue_submit": ([vp, vp, sz, ctypes.POINTER(ctypes.c_uint64)], i32),
            "lrb_queue_poll": ([vp, ctypes.c_uint64], i32),
            "lrb_queue_wait": ([vp, ctypes.c_uint64, ctypes.c_int], i32),
            "lrb_queue_latency": ([vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)], i32),
            "lrb_queue_stats": ([vp, ctypes.POINTER(lrb_queue_stats_t)], i32),
            "lrb_queue_destroy": ([vp, ctypes.c_int], i32),
            "lrb_split_dump_levels": ([vp, vp, vp], i32),
            "lrb_plan_tiles_host": ([vp, sz, i32, vp, sz, ctypes.POINTER(sz)], i32),
            "lrb_variant_count": ([], i32),
            "lrb_variant_shape": ([i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
            "lrb_execute_host_set_timing": ([vp, i32], i32),
            "lrb_execute_host_get_timing": ([vp, ctypes.POINTER(lrb_host_timing)], i32),
            "lrb_fp64_peak_probe": ([ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)], i32),
            "lrb_partition_lpt": ([vp, sz, i32, vp, vp], i32),
            "lrb_multi_plan_create": ([vp, i32, vp, sz, ctypes.POINTER(lrb_plan_opts), ctypes.POINTER(vp)], i32),
            "lrb_multi_launch": ([vp, vp], i32),
            "lrb_multi_plan_part": ([vp, i32, ctypes.POINTER(lrb_plan_info)], i32),
            "lrb_multi_plan_destroy": ([vp], i32),
            "lrb_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def declared_functions():
    """Names of the functions include/lrbatch.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lrb_\w+)\s*\(", text)))


def last_error() -> str:
    return lib().lrb_last_error().decode()


def check(status):
    if status != LRB_OK:
        raise LrbError(status, last_error())


def make_opts(precision=LRB_PREC_FP64, use_graph=False, tune=True, force_variant=-1, check_alias=True,
              test_stall=False, trans=0, overwrite=False):
    o = lrb_plan_opts()
    o.test_stall = int(bool(test_stall))
    o.trans = int(trans)
    o.overwrite = int(bool(overwrite))
    o.precision = precision
    o.use_graph = int(bool(use_graph))
    o.tune = int(bool(tune))
    o.force_variant = force_variant
    o.check_alias = int(bool(check_alias))
    return o


def descs_for(batch) -> np.ndarray:
    """Descriptor array for a workloads.Batch whose buffers are tensors."""
    d = np.zeros(len(batch), dtype=DESC_DTYPE)
    d["A"] = np.uint64(batch.A.data_ptr()) + 8 * batch.offA.astype(np.uint64)
    d["B"] = np.uint64(batch.B.data_ptr()) + 8 * batch.offB.astype(np.uint64)
    d["C"] = np.uint64(batch.C.data_ptr()) + 8 * batch.offC.astype(np.uint64)
    for key in ("m", "n", "k", "lda", "ldb", "ldc"):
        d[key] = getattr(batch, key)
    return d


def lr_descs_for(lb) -> np.ndarray:
    """lrb_lr_desc rows for a workloads.LrBatch whose buffers are tensors."""
    d = np.zeros(len(lb), dtype=LR_DESC_DTYPE)
    for key in ("AVT", "BU", "AX", "BX", "G"):
        d[key] = np.uint64(lb.bufs[key].data_ptr()) + 8 * lb.offs[key].astype(np.uint64)
    d["ra"], d["rb"], d["k"] = lb.ra, lb.rb, lb.k
    d["ld_avt"], d["ld_bu"], d["ld_ax"], d["ld_bx"], d["ldg"] = (lb.ra + lb.pad, lb.k + lb.pad, lb.ra + lb.pad,
                                                                 lb.rb + lb.pad, lb.ra + lb.pad)
    return d


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def lrb_validate(descs: np.ndarray, opts=None) -> int:
    descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    return lib().lrb_validate(descs.ctypes.data if len(descs) else None, len(descs),
                              ctypes.byref(opts) if opts is not None else None)


def lrb_plan_tiles_host(descs: np.ndarray, variant: int) -> np.ndarray:
    descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    n = ctypes.c_size_t(0)
    check(lib().lrb_plan_tiles_host(descs.ctypes.data, len(descs), variant, None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, 5), dtype=np.int32)
    check(lib().lrb_plan_tiles_host(descs.ctypes.data, len(descs), variant, out.ctypes.data, n.value,
                                    ctypes.byref(n)))
    return out


NOALLOC_MAX_ENTRIES = 4096      # LRB_NOALLOC_MAX_ENTRIES
NOALLOC_MAX_TILES = 262144      # LRB_NOALLOC_MAX_TILES


def lrb_launch_noalloc(descs: np.ndarray, stream=None) -> int:
    """lrb_launch_noalloc: the batch as one persistent FP64 launch that
    allocates no device memory (its scratch is a fixed array inside the
    library).  For callers that cannot call cudaMalloc -- e.g. their GPU
    memory belongs to a framework pool or a fixed budget, or their loop must
    not risk the device-wide synchronisation an allocation can cause.
    Returns the status code."""
    d = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    return lib().lrb_launch_noalloc(d.ctypes.data if len(d) else None, len(d), _stream_ptr(stream))


def lrb_partition_lpt(cost, parts: int):
    """Longest-processing-time partition (host only): (part of each item,
    total cost of each part)."""
    c = np.ascontiguousarray(cost, dtype=np.float64)
    part = np.zeros(len(c), dtype=np.int32)
    load = np.zeros(max(parts, 1), dtype=np.float64)
    check(lib().lrb_partition_lpt(c.ctypes.data if len(c) else None, len(c), int(parts), part.ctypes.data,
                                  load.ctypes.data))
    return part, load


class MultiPlan:
    """lrb_multi_plan_create / lrb_multi_launch / lrb_multi_plan_destroy: one
    batch partitioned (LPT over 2 m n k) across several handles, one plan per
    handle, launched with no synchronisation between the parts."""

    def __init__(self, handles, descs: np.ndarray, **opts):
        self.descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
        self.opts = make_opts(**opts)
        self.n = len(handles)
        arr = (ctypes.c_void_p * self.n)(*[h.ptr.value for h in handles])
        self.ptr = ctypes.c_void_p()
        check(lib().lrb_multi_plan_create(arr, self.n, self.descs.ctypes.data, len(self.descs), ctypes.byref(self.opts),
                                          ctypes.byref(self.ptr)))

    def launch(self, streams=None):
        if streams is None:
            check(lib().lrb_multi_launch(self.ptr, None))
            return
        arr = (ctypes.c_void_p * self.n)(*[_stream_ptr(s).value for s in streams])
        check(lib().lrb_multi_launch(self.ptr, arr))

    def part_info(self, i: int) -> dict:
        info = lrb_plan_info()
        check(lib().lrb_multi_plan_part(self.ptr, i, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in lrb_plan_info._fields_}

    def close(self):
        if self.ptr:
            check(lib().lrb_multi_plan_destroy(self.ptr))
            self.ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def lrb_fp64_peak_probe(device: int = 0, iters: int = 1 << 20):
    """Measured FP64-pipe throughput: (TFLOP/s, ms of the timed launch)."""
    t, ms = ctypes.c_double(0), ctypes.c_double(0)
    check(lib().lrb_fp64_peak_probe(device, int(iters), ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def lrb_variant_count() -> int:
    return lib().lrb_variant_count()


def lrb_variant_shape(v: int):
    bm, bn, dm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(lib().lrb_variant_shape(v, ctypes.byref(bm), ctypes.byref(bn), ctypes.byref(dm)))
    return bm.value, bn.value, bool(dm.value)


class Handle:
    """lrb_create / lrb_destroy."""

    def __init__(self, device: int = 0):
        self.ptr = ctypes.c_void_p()
        check(lib().lrb_create(ctypes.byref(self.ptr), device))

    def close(self):
        if self.ptr:
            check(lib().lrb_destroy(self.ptr))
            self.ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def plan(self, descs, **kw) -> "Plan":
        return Plan(self, descs, **kw)

    def execute_host(self, host_descs: np.ndarray, stream=None, **opts):
        """lrb_execute_host: descriptors with HOST pointers; returns when host C holds the result."""
        d = np.ascontiguousarray(host_descs, dtype=DESC_DTYPE)
        o = make_opts(**opts)
        check(lib().lrb_execute_host(self.ptr, d.ctypes.data, len(d), ctypes.byref(o), _stream_ptr(stream)))

    def set_host_timing(self, enable: bool = True):
        """lrb_execute_host_set_timing: record per-piece copy/launch intervals."""
        check(lib().lrb_execute_host_set_timing(self.ptr, int(bool(enable))))

    def host_timing(self) -> dict:
        """lrb_execute_host_get_timing: summary of the last timed execute_host call."""
        t = lrb_host_timing()
        check(lib().lrb_execute_host_get_timing(self.ptr, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in lrb_host_timing._fields_}


class Plan:
    """lrb_plan_create / lrb_launch / lrb_launch_plain / lrb_plan_destroy
    (lrb_lr_plan_create when lr_fused is given: descs are lrb_lr_desc rows)."""

    def __init__(self, handle: Handle, descs: np.ndarray, lr_fused=None, **opts):
        self.handle = handle
        self.ptr = ctypes.c_void_p()
        if lr_fused is not None:
            self.descs = np.ascontiguousarray(descs, dtype=LR_DESC_DTYPE)
            check(lib().lrb_lr_plan_create(handle.ptr, self.descs.ctypes.data, len(self.descs), int(bool(lr_fused)),
                                           ctypes.byref(self.ptr)))
            return
        self.descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
        self.opts = make_opts(**opts)
        check(lib().lrb_plan_create(handle.ptr, self.descs.ctypes.data, len(self.descs), ctypes.byref(self.opts),
                                    ctypes.byref(self.ptr)))

    def launch(self, stream=None):
        check(lib().lrb_launch(self.ptr, _stream_ptr(stream)))

    def launch_plain(self, stream=None):
        check(lib().lrb_launch_plain(self.ptr, _stream_ptr(stream)))

    def status(self) -> int:
        """lrb_plan_status: synchronises and reports an expired device wait."""
        return lib().lrb_plan_status(self.ptr)

    def dump_levels(self, dump_ptr: int, stream=None):
        check(lib().lrb_split_dump_levels(self.ptr, ctypes.c_void_p(dump_ptr), _stream_ptr(stream)))

    def info(self) -> dict:
        i = lrb_plan_info()
        check(lib().lrb_plan_get_info(self.ptr, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in lrb_plan_info._fields_}

    def close(self):
        if self.ptr:
            check(lib().lrb_plan_destroy(self.ptr))
            self.ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class LowRankPlan(Plan):
    """lrb_rsvd_plan_create / lrb_expand_plan_create / lrb_round_add_plan_create:
    kind "rsvd" (descs: RSVD_DESC_DTYPE rows, power_iters), "expand"
    (EXPAND_DESC_DTYPE) or "round_add" (ROUND_ADD_DESC_DTYPE).  Launch,
    status, info and close as for Plan."""

    _KINDS = {"rsvd": RSVD_DESC_DTYPE, "expand": EXPAND_DESC_DTYPE, "round_add": ROUND_ADD_DESC_DTYPE}

    def __init__(self, handle: Handle, kind: str, descs: np.ndarray, power_iters: int = 0):
        self.handle = handle
        self.ptr = ctypes.c_void_p()
        self.descs = np.ascontiguousarray(descs, dtype=self._KINDS[kind])
        d = self.descs.ctypes.data if len(self.descs) else None
        if kind == "rsvd":
            st = lib().lrb_rsvd_plan_create(handle.ptr, d, len(self.descs), int(power_iters), ctypes.byref(self.ptr))
        elif kind == "expand":
            st = lib().lrb_expand_plan_create(handle.ptr, d, len(self.descs), ctypes.byref(self.ptr))
        else:
            st = lib().lrb_round_add_plan_create(handle.ptr, d, len(self.descs), ctypes.byref(self.ptr))
        check(st)


class Queue:
    """lrb_queue_*: continuous-batching request queue on one handle."""

    def __init__(self, handle: Handle, budget_bytes: int, max_inflight: int = 4):
        self.ptr = ctypes.c_void_p()
        check(lib().lrb_queue_create(handle.ptr, int(budget_bytes), max_inflight, ctypes.byref(self.ptr)))

    def set_limits(self, max_waiting: int, max_wave_entries: int = 1 << 16):
        check(lib().lrb_queue_set_limits(self.ptr, max_waiting, max_wave_entries))

    def set_precision(self, precision: int):
        check(lib().lrb_queue_set_precision(self.ptr, precision))

    def submit(self, descs: np.ndarray):
        """Returns (status, ticket); status is LRB_OK, LRB_ERR_BUDGET, LRB_ERR_QUEUE_FULL or LRB_ERR_INVALID."""
        d = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
        t = ctypes.c_uint64(0)
        st = lib().lrb_queue_submit(self.ptr, d.ctypes.data if len(d) else None, len(d), ctypes.byref(t))
        return st, t.value

    def poll(self, ticket: int) -> int:
        return lib().lrb_queue_poll(self.ptr, ticket)

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        return lib().lrb_queue_wait(self.ptr, ticket, timeout_ms)

    def latency(self, ticket: int) -> float:
        v = ctypes.c_double(0)
        check(lib().lrb_queue_latency(self.ptr, ticket, ctypes.byref(v)))
        return v.value

    def stats(self) -> dict:
        s = lrb_queue_stats_t()
        check(lib().lrb_queue_stats(self.ptr, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in lrb_queue_stats_t._fields_}

    def close(self, timeout_ms: int = -1) -> int:
        st = LRB_OK
        if self.ptr:
            st = lib().lrb_queue_destroy(self.ptr, timeout_ms)
            self.ptr = ctypes.c_void_p()
        return st

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
