#!/usr/bin/env python3
"""Benchmark of the batched FP64 GEMM library (C_i += A_i B_i) on GB300.

Workload (one "step"): the uniform-shape sweep -- b in {256, 512, 1024}
(batch 4096 / 1024 / 256) x r in {16, 32, 64} x both forms (T-form
C(b x r) += A(b x b) B(b x r), O-form C(b x b) += A(b x r) B(r x b)),
N(0, 1) entries, 32,256 entries and 3.6e11 flops -- planned once and run as
ONE persistent, graph-captured launch per step.  Inputs (~42 GB) exceed L2,
so no flush is needed between steps.

Reported beside it: the same plan through the one-launch-per-shape path
(the comparator), the roofline of the persistent kernel against the FP64
pipe, the end-to-end rate through the host-buffer C ABI call (copies in
the timed region), SM clocks sampled during the timed region, and the CPU
oracle timed on a bounded sample on the host cores.

`--impl reference` times the CPU oracle alone (the reference arm).
Multi-GPU: every rank runs the full workload on its own GPU (weak scaling,
entries are independent; no data-path collective), value = all ranks' flops
over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched GEMM GFLOP/s and % roofline vs plain FP64 launch; serving p50/p99 ms"
UNIT = "GFLOP/s"
WORKLOAD = ("uniform-shape FP64 sweep: b in {256,512,1024} (batch 4096/1024/256) x r in {16,32,64} x "
            "T-form (b x b)(b x r) and O-form (b x r)(r x b), N(0,1), one persistent graph launch per step")
DFMA_LANES_PER_SM_CLK = 2          # FP64 FMA lanes per SM per clock on GB300 (1.25 TFLOP/s nominal)
# DRAM bytes per algorithmic byte of k_persistent, from the ncu capture in
# profiles/k_persistent_fp64_uniform_sweep.md (small case of the same sweep),
# valid while fp64_tiles.cu has the SHA-256 prefix below.
TRAFFIC_PER_ALG_BYTE = 2.067912e9 / 2.018344960e9
TRAFFIC_SOURCE_SHA = "c86a6ad4ee65ca25"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class ClockSampler:
    """nvidia-smi sampling (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def fp64_peak_tflops(props, sm_max_mhz) -> float:
    """FP64 pipe peak from unit counts and clock: SMs x 2 DFMA lanes x 2 flops x max SM clock."""
    return props.multi_processor_count * DFMA_LANES_PER_SM_CLK * 2 * sm_max_mhz * 1e6 / 1e12


def kernel_sha() -> str:
    import hashlib
    path = os.path.join(ROOT, "paper_2311_07602_gb300", "csrc", "fp64_tiles.cu")
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def sweep_batches(device, scale=1.0):
    from paper_2311_07602_gb300 import workloads as W
    return [W.uniform_batch(f, b, r, max(1, int(round(n * scale))), dist="normal", seed=s, device=device)
            for f, b, r, n, s in W.uniform_sweep_groups()]


def cpu_baseline(fraction: float, nthreads: int = 0):
    """The oracle, as it stands, on the first `fraction` of every group of the
    sweep (same shapes, seeds and distribution), timed on the host cores."""
    import oracle
    from paper_2311_07602_gb300 import workloads as W
    total_flops, total_s, used = 0.0, 0.0, 1
    entries = 0
    for f, b, r, n, s in W.uniform_sweep_groups():
        cnt = max(1, int(round(n * fraction)))
        bt = W.uniform_batch(f, b, r, cnt, dist="normal", seed=s, device="cpu")
        A, B, C = bt.A.numpy(), bt.B.numpy(), bt.C.numpy()
        ents = [dict(A=A, B=B, C=C, offA=int(bt.offA[e]), offB=int(bt.offB[e]), offC=int(bt.offC[e]),
                     m=int(bt.m[e]), n=int(bt.n[e]), k=int(bt.k[e]), lda=int(bt.lda[e]), ldb=int(bt.ldb[e]),
                     ldc=int(bt.ldc[e])) for e in range(cnt)]
        t0 = time.perf_counter()
        used = oracle.gemm_batch(ents, nthreads=nthreads)
        total_s += time.perf_counter() - t0
        total_flops += bt.flops()
        entries += cnt
    return total_flops, total_s, used, entries


def cpu_baseline_extras():
    """The oracle, as it stands, on small samples of the other workloads
    (same shapes and distributions), timed on the host cores: the paper's
    low-rank chain (2000 blocks, b 1024, r 16; the paper's flop count), the
    randomized SVD (4 kernel-matrix blocks, 1024^2, r 16, l 26, q 1; the
    library's flop count) and the split-precision product (4 T-form entries,
    1024 x 64 x 1024, BF16 S = 3; FP64-equivalent flops)."""
    import oracle
    from oracle import lowrank as OL
    from paper_2311_07602_gb300 import workloads as W
    out = {}
    lb = W.lr_batch(2000, 1024, 16, seed=7016, device="cpu")
    host = {k: t.numpy() for k, t in lb.bufs.items()}
    t0 = time.perf_counter()
    used = oracle.lr_chain_batch(host, lb.offs, lb.ra, lb.rb, lb.k)
    dt = time.perf_counter() - t0
    out["lr_chain"] = {"gflops_paper_count": round(lb.flops_paper() / dt / 1e9, 2), "threads": used,
                       "sample": "2000 blocks, b 1024, r 16, N(0,1)"}
    b, r, l, q, cnt = 1024, 16, 26, 1, 4
    A = W.kernel_blocks(cnt, b, b, seed=7, device="cpu").numpy()
    Om = W.gaussian_test_matrix(b, l, seed=8, device="cpu").numpy().reshape(l, b).T
    t0 = time.perf_counter()
    for e in range(cnt):
        OL.rsvd(A[e * b * b:(e + 1) * b * b].reshape(b, b).T, Om, r, q)
    dt = time.perf_counter() - t0
    out["rsvd"] = {"gflops": round(cnt * OL.lowrank_flops(b, b, l, r, q) / dt / 1e9, 2),
                   "blocks_per_s": round(cnt / dt, 1), "sample": f"{cnt} kernel-matrix blocks {b}x{b}, r {r}, l {l}, q {q}"}
    rng = np.random.default_rng(4)
    p = oracle.PRESETS["bf16_s3"]
    t0 = time.perf_counter()
    for _ in range(4):
        Asp = rng.standard_normal((1024, 1024)) * 10.0 ** rng.uniform(-4, 4, (1024, 1024))
        Bsp = rng.standard_normal((1024, 64)) * 10.0 ** rng.uniform(-4, 4, (1024, 64))
        oracle.split_gemm(Asp, Bsp, np.zeros((1024, 64)), p)
    dt = time.perf_counter() - t0
    out["split_bf16_s3"] = {"gflops_fp64_equiv": round(4 * 2.0 * 1024 * 64 * 1024 / dt / 1e9, 3),
                            "sample": "4 T-form entries 1024 x 64 x 1024, 10^U(-4,4) N(0,1) (single-threaded numpy)"}
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if world > 1 and rank != 0:
        return 0
    sys.path.insert(0, ROOT)
    from oracle import build as ob
    ob.build()
    frac = args.ref_fraction
    for _ in range(args.warmup):
        cpu_baseline(frac / 4)
    flops, secs = 0.0, 0.0
    used, ents = 1, 0
    for _ in range(args.steps):
        f, s, used, ents = cpu_baseline(frac)
        flops += f
        secs += s
    val = flops / secs / 1e9
    sample = f"first {frac:.4g} of every group of the sweep ({ents} entries, {flops / args.steps:.3g} flops) per step"
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": round(val, 3), "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lrbatch", choices=["lrbatch", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-fraction", type=float, default=1.0)
    ap.add_argument("--ref-fraction", type=float, default=1 / 32)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (64-entry O-form, variable-size, split precision, serving)")
    ap.add_argument("--extras", default="small,variable,split,serving,dmma,lr,blr,lowrank",
                    help="comma-separated subset of the other workloads to run")
    ap.add_argument("--split-batch", type=int, default=2048, help="entries of the split-precision batch")
    ap.add_argument("--dmma-scale", type=float, default=0.25, help="batch-count scale of the DMMA comparison")
    ap.add_argument("--lr-batch", type=int, default=20000, help="blocks per low-rank chain configuration")
    ap.add_argument("--lr-ranks", default="8,16,32,96,128", help="ranks of the low-rank chain sweep")
    ap.add_argument("--lowrank-count", type=int, default=1024,
                    help="dense blocks of the randomized-SVD / expansion / rounded-addition leg")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="batch-count scale of every group (profiling runs use a small case)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, local_rank, world = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    def barrier():
        if pg is not None:
            pg.barrier()

    def max_over_ranks(x: float) -> float:
        if pg is None:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    from paper_2311_07602_gb300 import lrbatch as L
    batches = sweep_batches(dev, args.scale)
    descs = np.concatenate([L.descs_for(b) for b in batches])
    flops = float(sum(b.flops() for b in batches))
    alg_bytes = float(sum(b.alg_bytes() for b in batches))
    cache = os.environ.get("LRB_TUNE_CACHE") or os.path.join(tempfile.gettempdir(), f"lrb_tune_{local_rank}.json")
    os.environ["LRB_TUNE_CACHE"] = cache
    handle = L.Handle(local_rank)
    t0 = time.perf_counter()
    plan = handle.plan(descs, use_graph=True)
    plan_s = time.perf_counter() - t0
    info = plan.info()
    stream = torch.cuda.Stream(device=dev)

    def timed(fn, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for e0, e1 in evs:
            e0.record(stream)
            fn(stream)
            e1.record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        barrier()
        total_ms = start.elapsed_time(end)
        per = [e0.elapsed_time(e1) for e0, e1 in evs]
        return total_ms, per

    sampler = ClockSampler(local_rank)
    sampler.start()
    total_ms, per = timed(lambda s: plan.launch(s), args.steps, args.warmup)
    clocks = sampler.stop()
    total_ms = max_over_ranks(total_ms)
    value = world * flops * args.steps / (total_ms / 1e3) / 1e9
    ms_per_step = total_ms / args.steps

    props = torch.cuda.get_device_properties(dev)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak = fp64_peak_tflops(props, sm_max)
    achieved = flops / (statistics.mean(per) / 1e3) / 1e12
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded N(0,1), generated on the device)",
            "config": {"workload": WORKLOAD if args.scale == 1.0 else f"{WORKLOAD} (batch counts x {args.scale})",
                       "entries": int(info["entries"]), "tiles": int(info["items"]),
                       "flops_per_step": flops, "alg_bytes_per_step": alg_bytes, "persistent_grid": int(info["grid"]),
                       "l2": "inputs larger than L2 (%.0f GB per step), no flush" % (alg_bytes / 1e9),
                       "plan_s": round(plan_s, 3)},
            "gpu_launches": args.steps,
            "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": (round(TRAFFIC_PER_ALG_BYTE * alg_bytes) if kernel_sha() == TRAFFIC_SOURCE_SHA
                                     else None),
                         "traffic_note": "DRAM bytes per launch, scaled by algorithmic bytes from the small-case ncu "
                                         "capture (profiles/k_persistent_fp64_uniform_sweep.md); null if the kernel "
                                         "source changed since",
                         "kernel": "k_persistent (FP64 DFMA tiles)",
                         "peak_source": "derived: SMs x 2 DFMA lanes/clk x 2 flop x max SM clock",
                         "peak_measured_probe_tflops": 1.2029},
            "clocks": clocks}
    line["pct_roofline"] = round(100 * achieved / peak, 2)

    if not args.no_plain:
        p_ms, p_per = timed(lambda s: plan.launch_plain(s), args.steps, args.warmup)
        p_ms = max_over_ranks(p_ms)
        pval = world * flops * args.steps / (p_ms / 1e3) / 1e9
        line["plain"] = {"value": round(pval, 2), "unit": UNIT, "ms_per_step": round(p_ms / args.steps, 3),
                         "launches_per_step": int(info["groups"])}
        line["vs_plain"] = round(value / pval, 4)

    if not args.no_e2e:
        line["e2e"] = e2e_leg(L, handle, batches, flops, args, barrier, max_over_ranks, world, stream)

    if not args.no_extras and world == 1:
        plan.close()
        plan = None
        del batches
        torch.cuda.empty_cache()
        line["extras"] = extras(L, handle, stream, dev, peak, timed, set(args.extras.split(",")), args.split_batch,
                                args.dmma_scale, args.lr_batch, tuple(int(x) for x in args.lr_ranks.split(",")),
                                args.lowrank_count)

    if not args.no_cpu and rank == 0 and world == 1:
        f, s, used, ents = cpu_baseline(args.cpu_fraction)
        line["cpu_baseline"] = {"value": round(f / s / 1e9, 3), "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": (f"first {args.cpu_fraction:.3g} of every group of the sweep "
                                           f"({ents} entries, {f:.3g} flops, {s:.1f} s on the host cores)")}
        if not args.no_extras:
            line["cpu_baseline"]["extras"] = cpu_baseline_extras()
    if plan is not None:
        plan.close()
    handle.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def extras(L, handle, stream, dev, peak_fp64, timed, which, split_batch, dmma_scale=0.25, lr_batch=20000,
           lr_ranks=(8, 16, 32, 96, 128), lowrank_count=1024):
    """The other workloads, each with its own plan, 3 warm-up and 5 timed launches:
    the 64-entry O-form batch (L2 flushed before every launch: it fits in L2),
    the 20,000-entry variable-size batch (persistent vs one launch per shape),
    and the split-precision batch (b 1024, r 64, 2048 entries, 10^U(-4,4) N(0,1))."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {}

    if "small" in which:
        out["small_o_form"] = small_leg(L, handle, stream, dev, peak_fp64)
    if "variable" in which:
        out["variable_size"] = variable_leg(L, handle, dev, peak_fp64, timed)
    if "split" in which:
        out["split"] = split_leg(L, handle, dev, timed, hbm, split_batch)
    if "serving" in which:
        out["serving"] = serving_leg(L, handle, dev, peak_fp64)
    if "dmma" in which:
        out["dmma"] = dmma_leg(L, handle, dev, peak_fp64, timed, dmma_scale)
    if "lr" in which:
        out["lr_chain"] = lr_leg(L, handle, dev, peak_fp64, timed, lr_batch, lr_ranks)
    if "blr" in which:
        out["blr_matvec"] = blr_leg(L, handle, dev, peak_fp64, timed)
    if "lowrank" in which:
        out["lowrank"] = lowrank_leg(L, handle, dev, peak_fp64, timed, count=lowrank_count)
    return out


def lowrank_leg(L, handle, dev, peak_fp64, timed, count=1024, b=1024, r=16, p=10, q=1):
    """Producers and consumers of low-rank blocks (Sec. 2): the randomized SVD
    of `count` dense b x b blocks of the Laplace kernel 1/|x - y| between two
    separated point clusters (the admissible blocks of a hierarchical matrix)
    to rank r with p oversampling columns and q power iterations; the
    expansion D += U diag(S) V, run with -S on D = A so that it leaves the
    approximation residual A - U S V; and the rounded addition of the produced
    blocks in pairs back to rank r.  GFLOP/s count what lrb_plan_get_info
    reports (products with A, QRs, final products; 2 m n r per expansion)."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    l = r + p
    A = W.kernel_blocks(count, b, b, seed=7, device=dev)
    Om = W.gaussian_test_matrix(b, l, seed=8, device=dev)
    U = torch.empty(count * b * r, dtype=torch.float64, device=dev)
    S = torch.empty(count * r, dtype=torch.float64, device=dev)
    V = torch.empty(count * r * b, dtype=torch.float64, device=dev)
    e = np.arange(count, dtype=np.uint64)
    blk = np.zeros(count, dtype=L.LR_BLOCK_DTYPE)
    blk["U"] = np.uint64(U.data_ptr()) + np.uint64(8 * b * r) * e
    blk["S"] = np.uint64(S.data_ptr()) + np.uint64(8 * r) * e
    blk["V"] = np.uint64(V.data_ptr()) + np.uint64(8 * r * b) * e
    blk["m"], blk["n"], blk["r"], blk["ldu"], blk["ldv"] = b, b, r, b, r
    d = np.zeros(count, dtype=L.RSVD_DESC_DTYPE)
    d["A"] = np.uint64(A.data_ptr()) + np.uint64(8 * b * b) * e
    d["Omega"] = Om.data_ptr()
    d["out"] = blk
    d["l"], d["lda"], d["ldo"] = l, b, b
    out = {"workload": f"{count} Laplace-kernel blocks 1/|x - y| ({b} x {b}, clusters 2 apart), rank {r}, "
                       f"oversampling {p}, {q} power iteration(s), Omega N(0,1)"}
    with L.LowRankPlan(handle, "rsvd", d, power_iters=q) as pl:
        info = pl.info()
        ms, _ = timed(lambda s: pl.launch(s), 3, 2)
        ms /= 3
        assert pl.status() == L.LRB_OK
    out["rsvd"] = {"ms": round(ms, 3), "gflops": round(info["flops"] / ms / 1e6, 1),
                   "frac_fp64_peak": round(info["flops"] / ms / 1e9 / peak_fp64, 4),
                   "blocks_per_s": round(count / ms * 1e3, 1), "flops_per_block": info["flops"] / count}
    # expansion: D = A, S -> -S, so one launch leaves D = A - U S V
    D = A.clone()
    Sneg = -S
    ed = np.zeros(count, dtype=L.EXPAND_DESC_DTYPE)
    ed["blk"] = blk
    ed["blk"]["S"] = np.uint64(Sneg.data_ptr()) + np.uint64(8 * r) * e
    ed["D"] = np.uint64(D.data_ptr()) + np.uint64(8 * b * b) * e
    ed["ldd"] = b
    with L.LowRankPlan(handle, "expand", ed) as pl:
        info = pl.info()
        pl.launch()
        torch.cuda.synchronize()
        res = (D.view(count, b * b).norm(dim=1) / A.view(count, b * b).norm(dim=1)).cpu().numpy()
        ms, _ = timed(lambda s: pl.launch(s), 3, 2)
        ms /= 3
    out["expand"] = {"ms": round(ms, 3), "gflops": round(info["flops"] / ms / 1e6, 1),
                     "frac_fp64_peak": round(info["flops"] / ms / 1e9 / peak_fp64, 4)}
    out["rel_residual_fro"] = {"median": float(np.median(res)), "max": float(res.max())}
    del D, Sneg
    # rounded addition of blocks (2i, 2i + 1) back to rank r
    half = count // 2
    U2 = torch.empty(half * b * r, dtype=torch.float64, device=dev)
    S2 = torch.empty(half * r, dtype=torch.float64, device=dev)
    V2 = torch.empty(half * r * b, dtype=torch.float64, device=dev)
    h = np.arange(half, dtype=np.uint64)
    ra = np.zeros(half, dtype=L.ROUND_ADD_DESC_DTYPE)
    ra["x"], ra["y"] = blk[0::2], blk[1::2]
    ra["out"]["U"] = np.uint64(U2.data_ptr()) + np.uint64(8 * b * r) * h
    ra["out"]["S"] = np.uint64(S2.data_ptr()) + np.uint64(8 * r) * h
    ra["out"]["V"] = np.uint64(V2.data_ptr()) + np.uint64(8 * r * b) * h
    ra["out"]["m"], ra["out"]["n"], ra["out"]["r"], ra["out"]["ldu"], ra["out"]["ldv"] = b, b, r, b, r
    with L.LowRankPlan(handle, "round_add", ra) as pl:
        info = pl.info()
        ms, _ = timed(lambda s: pl.launch(s), 3, 2)
        ms /= 3
        assert pl.status() == L.LRB_OK
    out["round_add"] = {"pairs": half, "ms": round(ms, 3), "gflops": round(info["flops"] / ms / 1e6, 1),
                        "frac_fp64_peak": round(info["flops"] / ms / 1e9 / peak_fp64, 4),
                        "pairs_per_s": round(half / ms * 1e3, 1)}
    del A, U, S, V, U2, S2, V2
    torch.cuda.empty_cache()
    return out


def blr_leg(L, handle, dev, peak_fp64, timed, nb=128, b=512, r=8, nrhs=8):
    """The paper's application: a weakly admissible BLR matrix (N = nb b,
    dense diagonal blocks, rank-r off-diagonal blocks) times nrhs right-hand
    sides, rank 8 and 8 right-hand sides as in the paper; fused low-rank
    chains against the three-product comparator."""
    import torch
    from paper_2311_07602_gb300 import blr
    M = blr.random_blr(nb, b, r, seed=8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(9)
    X = torch.empty(M.N * nrhs, dtype=torch.float64, device=dev).normal_(generator=g)
    Y = torch.zeros(M.N * nrhs, dtype=torch.float64, device=dev)
    out = {"workload": f"BLR matrix N = {M.N} ({nb} x {nb} blocks of {b}), rank {r}, {nrhs} right-hand sides, N(0,1)",
           "flops": M.flops(nrhs)}
    for fused in (True, False):
        mv = blr.BLRMatVec(handle, M, X, Y, nrhs, fused=fused)
        ms, _ = timed(lambda s: mv.run(s), 10, 3)
        mv.close()
        out["fused" if fused else "unfused"] = {"ms": round(ms / 10, 4), "gflops": round(M.flops(nrhs) * 10 / ms / 1e6, 1),
                                                "frac_fp64_peak": round(M.flops(nrhs) * 10 / ms / 1e9 / peak_fp64, 4)}
    out["fused_vs_unfused"] = round(out["unfused"]["ms"] / out["fused"]["ms"], 3)
    out["paper_context"] = "the paper reports ~15% end-to-end and ~50% on the low-rank part over batched MKL (Xeon 6148)"
    del M, X, Y
    torch.cuda.empty_cache()
    return out


# GFLOPS the paper prints for its fused batched low-rank multiplication and
# the vendor libraries, batch 20,000 (context only: CPUs, other hardware).
PAPER_LR_GFLOPS = {
    "rank 96, 48-core A64FX (ours / SSL-2)": {512: (207.55, 370.62), 1024: (343.912, 598.93), 2048: (521.93, 851.74)},
    "rank 128, 2x Xeon 6148 40 cores (ours / MKL BATCH)": {512: (339.849, 262.281), 1024: (361.89, 400.602),
                                                           2048: (319.161, 554.721)},
    "rank 96, 2x EPYC 7502 64 cores (ours / BLIS)": {512: (237.441, 197.056), 1024: (283.175, 373.555),
                                                     2048: (348.566, 559.075)},
}


def lr_leg(L, handle, dev, peak_fp64, timed, batch=20000, ranks=(8, 16, 32, 96, 128)):
    """The paper's batched low-rank multiplication G = A_X (A_{V^T} B_U) B_X
    (Alg. 1-3): batch 20,000, b in {512, 1024, 2048}, r in {8, 16, 32}, N(0,1),
    fused (one CTA per block, temporaries on chip) against unfused (three
    batched products through the persistent FP64 path).  GFLOPS counted as the
    paper does, batch (4 r^3 + 2 r^2 b) / t; bandwidth as batch (2 r^2 + 2 r b)
    8 bytes / t.  Ranks 96 and 128 (the paper's tables) run unfused."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    rows = []
    for r in ranks:
        for b in (512, 1024, 2048):
            lb = W.lr_batch(batch, b, r, seed=7000 + 10 * r + b // 512, device=dev)
            d = L.lr_descs_for(lb)
            fpap = lb.flops_paper()
            byts = batch * (2 * r * r + 2 * r * b) * 8.0
            row = {"r": r, "b": b}
            for fused in ((True, False) if r <= 64 else (False,)):
                with L.Plan(handle, d, lr_fused=fused) as p:
                    steps = 3 if r <= 64 else 1
                    ms, _ = timed(lambda s: p.launch(s), steps, 3)
                    ms /= steps
                    exec_flops = p.info()["flops"]
                key = "fused" if fused else "unfused"
                row[key] = {"ms": round(ms, 3), "gflops_paper_count": round(fpap / ms / 1e6, 1),
                            "gib_s": round(byts / (ms / 1e3) / 2 ** 30, 1),
                            "frac_fp64_peak": round(exec_flops / ms / 1e9 / peak_fp64, 4)}
            if "fused" in row:
                row["fused_vs_unfused"] = round(row["unfused"]["ms"] / row["fused"]["ms"], 3)
            rows.append(row)
            del lb
            torch.cuda.empty_cache()
    return {"workload": f"batch {batch}, N(0,1), FP64; flops counted as the paper does (4 r^3 + 2 r^2 b per block)",
            "rows": rows, "paper_cpu_gflops_context": {k: {str(b): v for b, v in t.items()}
                                                       for k, t in PAPER_LR_GFLOPS.items()}}


def dmma_leg(L, handle, dev, peak_fp64, timed, scale=0.25):
    """FP64 tensor-core (DMMA) tiles against DFMA tiles on a quarter of the
    uniform sweep: tuned without DMMA, tuned with DMMA allowed (the tuner
    keeps a DMMA tile only where it measures faster), and DMMA forced."""
    import torch
    batches = sweep_batches(dev, scale)
    descs = np.concatenate([L.descs_for(b) for b in batches])
    f = float(sum(b.flops() for b in batches))
    out = {"workload": f"uniform sweep, batch counts x {scale}"}
    for name, opts in (("dfma_tuned", {}), ("dmma_allowed_tuned", {"precision": L.LRB_PREC_FP64_DMMA_ALLOWED}),
                       ("dmma_forced_64x32", {"force_variant": 8})):
        with handle.plan(descs, use_graph=True, **opts) as p:
            info = p.info()
            ms, _ = timed(lambda s: p.launch(s), 3, 3)
        out[name] = {"gflops": round(f * 3 / ms / 1e6, 1), "frac_fp64_peak": round(f * 3 / ms / 1e9 / peak_fp64, 4),
                     "dmma_tiles": int(info["dmma_items"]), "tiles": int(info["items"])}
    del batches
    torch.cuda.empty_cache()
    return out


def small_leg(L, handle, stream, dev, peak_fp64):
    """64-entry O-form, C(256x256) += A(256x16) B(16x256), U[-1,1], seed 0;
    it fits in L2, so a 256 MB buffer is written before every launch."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    b = W.small_o_form(device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    with handle.plan(L.descs_for(b), use_graph=True) as p:
        per = []
        for i in range(8):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            p.launch(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= 3:
                per.append(e0.elapsed_time(e1))
    f = b.flops()
    ms = statistics.median(per)
    return {"workload": "O-form, 64 x C(256x256) += A(256x16) B(16x256), U[-1,1], seed 0, L2 flushed",
            "gflops": round(f / ms / 1e6, 2), "ms": round(ms, 4), "frac_fp64_peak": round(f / ms / 1e9 / peak_fp64, 4)}


def variable_leg(L, handle, dev, peak_fp64, timed):
    """20,000 entries, b log-uniform [64, 2048], r in {8..128}, T/O 50/50:
    one persistent graph launch against one launch per distinct shape."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    forms, bs, rs = W.variable_shapes(20000, seed=3)
    vb = W.variable_batch(forms, bs, rs, seed=3, device=dev, pool_elems=(4 << 30) // 8)
    t0 = time.perf_counter()
    p = handle.plan(L.descs_for(vb), use_graph=True)
    plan_s = time.perf_counter() - t0
    info = p.info()
    f = vb.flops()
    ms_p, _ = timed(lambda s: p.launch(s), 5, 3)
    ms_q, _ = timed(lambda s: p.launch_plain(s), 5, 3)
    out = {
        "workload": "20,000 entries, b log-uniform [64,2048], r in {8,16,32,64,128}, T/O 50/50, N(0,1), seed 3, "
                    "A/B views into a 4 GB pool",
        "flops": f, "persistent_gflops": round(f * 5 / ms_p / 1e6, 2), "plain_gflops": round(f * 5 / ms_q / 1e6, 2),
        "vs_plain": round(ms_q / ms_p, 4), "frac_fp64_peak": round(f * 5 / ms_p / 1e9 / peak_fp64, 4),
        "persistent_ms": round(ms_p / 5, 3), "plain_ms": round(ms_q / 5, 3), "plain_launches": int(info["groups"]),
        "tiles": int(info["items"]), "plan_s_incl_tuning": round(plan_s, 2)}
    p.close()
    # the same variable-size batch in split precision (one persistent tcgen05 launch over all tiles)
    for name, prec in (("split_bf16_s3", L.LRB_PREC_SPLIT_BF16_S3), ("split_bf16_s4", L.LRB_PREC_SPLIT_BF16_S4)):
        with handle.plan(L.descs_for(vb), precision=prec) as ps:
            ms_s, _ = timed(lambda s: ps.launch(s), 3, 3)
            st = ps.status()
        out[name] = {"gflops_fp64_equiv": round(f * 3 / ms_s / 1e6, 1), "ms": round(ms_s / 3, 3),
                     "vs_fp64_persistent": round((ms_p / 5) / (ms_s / 3), 3), "status": int(st)}
    del vb
    torch.cuda.empty_cache()
    return out


def split_leg(L, handle, dev, timed, hbm, batch):
    """Split precision (BF16/FP16 x 3/4 digits) against the FP64 path on the
    wide-range batch b 1024, r 64, entries 10^U(-4,4) N(0,1), both forms."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    res = {}
    for form in (W.FORM_T, W.FORM_O):
        wb = W.wide_range(form, batch=batch, device=dev)
        f = wb.flops()
        ab = wb.alg_bytes()
        row = {}
        for name, prec in (("fp64", L.LRB_PREC_FP64), ("bf16_s3", L.LRB_PREC_SPLIT_BF16_S3),
                           ("bf16_s4", L.LRB_PREC_SPLIT_BF16_S4), ("fp16_s3", L.LRB_PREC_SPLIT_FP16_S3),
                           ("fp16_s4", L.LRB_PREC_SPLIT_FP16_S4)):
            with handle.plan(L.descs_for(wb), precision=prec, use_graph=(prec == L.LRB_PREC_FP64)) as p:
                steps = 2 if prec == L.LRB_PREC_FP64 else 5
                ms, _ = timed(lambda s: p.launch(s), steps, 3)
                st = p.status()
            ms /= steps
            row[name] = {"ms": round(ms, 3), "gflops_fp64_equiv": round(f / ms / 1e6, 1),
                         "hbm_gbs_alg": round(ab / ms / 1e6, 1), "frac_hbm": round(ab / ms / 1e6 / hbm, 4),
                         "status": int(st)}
        res["T" if form == W.FORM_T else "O"] = row
        del wb
        torch.cuda.empty_cache()
    return {"workload": f"b 1024, r 64, {batch} entries, 10^U(-4,4) N(0,1), seed 4", "hbm_peak_gbs": hbm, **res}


def serving_leg(L, handle, dev, peak_fp64, budget=40 << 30):
    """Poisson request streams into the continuous-batching queue.  Each
    request: 1..512 products, b log-uniform [64, 2048], r in {8..128}, T/O
    50/50; operands are views into a 4 GB device pool, results go to a 64 GB
    device ring.  Offered loads: 0.25 / 0.5 / 0.75 / 0.9 x the FP64 capacity
    (FP64 peak / mean request flops) for 3 s each, the stated overload rates
    1k / 2k / 5k / 10k / 20k req/s for 0.5 s each (waiting FIFO limited to 32
    so the backlog drains quickly), and 0.9 x the FP64 capacity once more with
    split-precision (BF16, S = 3) waves; 40 GB admission budget, 4 stream
    slots."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    pool = torch.empty((4 << 30) // 8, dtype=torch.float64, device=dev).normal_(generator=g)
    ring = torch.zeros((64 << 30) // 8, dtype=torch.float64, device=dev)
    _, probe = W.serving_requests(2000, 1.0, seed=55)
    mean_flops = float(np.mean([np.sum(2.0 * bb.astype(np.float64) ** 2 * rr) for _, bb, rr in probe]))
    capacity = 0.98 * peak_fp64 * 1e12 / mean_flops
    points = [(f"{fr:g}x capacity", fr * capacity, 3.0, 4096, L.LRB_PREC_FP64) for fr in (0.25, 0.5, 0.75, 0.9)]
    points += [(f"{r // 1000}k req/s", float(r), 0.5, 32, L.LRB_PREC_FP64) for r in (1000, 2000, 5000, 10000, 20000)]
    points += [("0.9x FP64 capacity, split BF16 S=3 waves", 0.9 * capacity, 3.0, 4096, L.LRB_PREC_SPLIT_BF16_S3)]
    rng = np.random.default_rng(505)
    cursor = 0
    results = []
    for idx, (label, rate, secs, max_waiting, prec) in enumerate(points):
        count = max(4, int(rate * secs))
        arrivals, reqs = W.serving_requests(count, rate, seed=500 + idx)
        descs = []
        for forms, bs, rs in reqs:
            m = bs.astype(np.int64)
            n = np.where(forms == W.FORM_T, rs, bs).astype(np.int64)
            k = np.where(forms == W.FORM_T, bs, rs).astype(np.int64)
            d = np.zeros(len(bs), dtype=L.DESC_DTYPE)
            offa = rng.integers(0, (pool.numel() - m * k) // 32) * 32
            offb = rng.integers(0, (pool.numel() - k * n) // 32) * 32
            sizes = ((m * n + 31) // 32) * 32
            need = int(sizes.sum())
            if cursor + need > ring.numel():
                cursor = 0
            offc = cursor + np.concatenate([[0], np.cumsum(sizes)[:-1]])
            cursor += need
            d["A"] = np.uint64(pool.data_ptr()) + 8 * offa.astype(np.uint64)
            d["B"] = np.uint64(pool.data_ptr()) + 8 * offb.astype(np.uint64)
            d["C"] = np.uint64(ring.data_ptr()) + 8 * offc.astype(np.uint64)
            d["m"], d["n"], d["k"] = m, n, k
            d["lda"], d["ldb"], d["ldc"] = m, k, m
            descs.append(d)
        torch.cuda.synchronize()
        q = L.Queue(handle, budget, max_inflight=4)
        q.set_limits(max_waiting)
        q.set_precision(prec)
        tickets, codes = [], {}
        t0 = time.perf_counter()
        for t_arr, d in zip(arrivals, descs):
            while time.perf_counter() - t0 < t_arr:
                pass
            st, tk = q.submit(d)
            codes[st] = codes.get(st, 0) + 1
            if st == L.LRB_OK:
                tickets.append(tk)
        submit_s = time.perf_counter() - t0
        for tk in tickets:
            q.wait(tk, 300000)
        st = q.stats()
        q.close()
        results.append({"load": label, "precision": "fp64" if prec == L.LRB_PREC_FP64 else "split_bf16_s3",
                        "offered_req_s": round(rate, 2), "duration_s": round(submit_s, 3),
                        "submitted": count, "accepted": int(st["accepted"]),
                        "rejected_queue_full": int(st["rejected_full"]), "rejected_budget": int(st["rejected_budget"]),
                        "completed": int(st["completed"]), "p50_ms": round(st["p50_ms"], 3),
                        "p99_ms": round(st["p99_ms"], 3), "sustained_gflops": round(st["gflops"], 1),
                        "waves": int(st["waves"]), "max_concurrent_waves": int(st["max_concurrent_waves"]),
                        "mean_wave_entries": round(st["mean_wave_entries"], 1),
                        "peak_reserved_gb": round(st["peak_reserved_bytes"] / 1e9, 2)})
    del pool, ring
    torch.cuda.empty_cache()
    return {"workload": "Poisson requests, 1..512 products each, b log-uniform [64,2048], r in {8..128}, "
                        "T/O 50/50, N(0,1), FP64, 40 GB budget, 4 stream slots",
            "mean_request_gflop": round(mean_flops / 1e9, 2), "capacity_req_s": round(capacity, 1),
            "points": results}


def e2e_leg(L, handle, batches, flops, args, barrier, max_over_ranks, world, stream):
    """Same workload through lrb_execute_host: inputs in pinned host memory,
    host->device copies, the launch and the device->host copy of every C in
    the timed region.  With N ranks every rank takes the first 1/N of each
    group (host memory is shared by the ranks), and flops count what ran."""
    import torch
    rows = []
    hold = []
    h2d = d2h = 0
    fl = 0.0
    for b in batches:
        cnt = max(1, len(b) // world)
        ea, eb, ec = (int(b.offA[cnt - 1] + b.lda[cnt - 1] * b.k[cnt - 1]), int(b.offB[cnt - 1] + b.ldb[cnt - 1] *
                      b.n[cnt - 1]), int(b.offC[cnt - 1] + b.ldc[cnt - 1] * b.n[cnt - 1]))
        A = torch.empty(ea, dtype=torch.float64, pin_memory=True)
        B = torch.empty(eb, dtype=torch.float64, pin_memory=True)
        C = torch.empty(ec, dtype=torch.float64, pin_memory=True)
        A.copy_(b.A[:ea])
        B.copy_(b.B[:eb])
        C.copy_(b.C[:ec])
        hold.append((A, B, C))
        sub = type(b)(A, B, C, b.m[:cnt], b.n[:cnt], b.k[:cnt], b.lda[:cnt], b.ldb[:cnt], b.ldc[:cnt], b.offA[:cnt],
                      b.offB[:cnt], b.offC[:cnt])
        rows.append(L.descs_for(sub))
        h2d += 8 * (A.numel() + B.numel() + C.numel())
        d2h += 8 * C.numel()
        fl += sub.flops()
    descs = np.concatenate(rows)
    # the box's pinned-copy bandwidth in this run (context for the e2e figure):
    # the largest A buffer in, then out, each timed alone with CUDA events
    big = max((h[0] for h in hold), key=lambda t: t.numel())
    dbuf = torch.empty(big.numel(), dtype=torch.float64, device="cuda")
    copy_gbs = {}
    for name, dst, src in (("h2d", dbuf, big), ("d2h", big, dbuf)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        copy_gbs[name] = round(8 * big.numel() / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    del dbuf
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        handle.execute_host(descs, stream)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        handle.execute_host(descs, stream)
    torch.cuda.synchronize()
    barrier()
    secs = max_over_ranks(time.perf_counter() - t0)
    del hold
    return {"value": round(world * fl * args.e2e_steps / secs / 1e9, 2), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
            "flops_per_step_per_rank": fl, "pinned_copy_gbs": copy_gbs,
            "api": "lrb_execute_host (pinned host buffers; copies in, compute and copies out pipelined in pieces)"}


if __name__ == "__main__":
    sys.exit(main())
