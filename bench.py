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
TRAFFIC_PER_ALG_BYTE = 1.959e9 / 2.018344960e9
TRAFFIC_SOURCE_SHA = "90b6a78a72fcf2dc"


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

    if not args.no_cpu and rank == 0 and world == 1:
        f, s, used, ents = cpu_baseline(args.cpu_fraction)
        line["cpu_baseline"] = {"value": round(f / s / 1e9, 3), "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": (f"first {args.cpu_fraction:.3g} of every group of the sweep "
                                           f"({ents} entries, {f:.3g} flops, {s:.1f} s on the host cores)")}
    plan.close()
    handle.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def e2e_leg(L, handle, batches, flops, args, barrier, max_over_ranks, world, stream):
    """Same workload through lrb_execute_host: inputs in pinned host memory,
    host->device copies, the launch and the device->host copy of every C in
    the timed region."""
    import torch
    host = []
    rows = []
    h2d = d2h = 0
    for b in batches:
        A = torch.empty(b.A.numel(), dtype=torch.float64, pin_memory=True)
        B = torch.empty(b.B.numel(), dtype=torch.float64, pin_memory=True)
        C = torch.empty(b.C.numel(), dtype=torch.float64, pin_memory=True)
        A.copy_(b.A)
        B.copy_(b.B)
        C.copy_(b.C)
        host.append((A, B, C))
        d = L.descs_for(type(b)(A, B, C, b.m, b.n, b.k, b.lda, b.ldb, b.ldc, b.offA, b.offB, b.offC))
        rows.append(d)
        h2d += 8 * (A.numel() + B.numel() + C.numel())
        d2h += 8 * C.numel()
    descs = np.concatenate(rows)
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
    del host
    return {"value": round(world * flops * args.e2e_steps / secs / 1e9, 2), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
            "api": "lrb_execute_host (pinned host buffers)"}


if __name__ == "__main__":
    sys.exit(main())
