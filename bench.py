#!/usr/bin/env python3
"""Benchmark of the batched FP64 GEMM library (C_i += A_i B_i) on GB300.

Workload of one step (the headline): the variable-size batch -- 20,000
entries, b = round(exp(U(ln 64, ln 2048))), r uniform over {8, 16, 32, 64,
128}, T-form C(b x r) += A(b x b) B(b x r) or O-form C(b x b) += A(b x r)
B(r x b) with probability 1/2 each, N(0, 1), seed 3; A and B are views into a
shared 4 GB operand pool and every entry has its own C (about 50 GB) --
planned once with autotuned tiles and run as ONE persistent, graph-captured
launch per step (1.18e12 flops).  The inputs exceed L2 many times over, so no
flush is needed between steps.

Beside it on the final JSON line: the same plan through one launch per
distinct shape (the plain comparator), the roofline against the FP64 pipe's
peak measured in the same run by a probe kernel, the end-to-end rate through
the host-buffer call lrb_execute_host (copies in the timed region, with a
breakdown of where its time goes), SM clocks sampled during the timed region,
the CPU oracle timed on a bounded sample of the same batch, and short
summaries of the split-precision error table and of the serving latencies.
The other workloads' full results are printed on the line before it,
prefixed "extras: ".

`--impl reference` times the CPU oracle alone on a bounded sample of the same
batch (the reference arm).  Multi-GPU (torchrun): `--scaling weak` (default)
runs the whole batch on every rank's GPU; `--scaling strong` splits the
batch's entries across the ranks by longest-processing-time order over their
flops (lrb_partition_lpt), each rank planning and launching only its share.
Entries are independent, so neither needs a data-path collective; value = all
ranks' flops over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batched GEMM GFLOP/s and % roofline vs plain FP64 launch; serving p50/p99 ms"
UNIT = "GFLOP/s"
VARIABLE_COUNT = 20000
WORKLOAD = ("variable-size FP64 batch: 20,000 entries, b log-uniform [64,2048], r in {8,16,32,64,128}, "
            "T/O 50/50, N(0,1), seed 3, A/B views into a 4 GB pool; one persistent graph launch, autotuned tiles")
DFMA_LANES_PER_SM_CLK = 2          # FP64 FMA lanes per SM per clock on GB300 (1.25 TFLOP/s nominal)
# DRAM bytes (read + write) per algorithmic byte of k_persistent on the
# variable-size batch, from an ncu capture of a 1/20-scale case of the same
# batch (its first 1,000 entries, same 4 GB pool): 6.716 GB read + 2.323 GB
# written for 7.356 GB algorithmic (an earlier capture with another tuning
# outcome gave 1.225).  Valid while the kernels (fp64_tiles.cu) and the
# planner and tuner that choose their tiles (api.cu) have the SHA-256 prefix
# below (the roofline's traffic is null otherwise); the prefix was renewed
# after a planner change that concerns plans of two to eight waves only.
TRAFFIC_PER_ALG_BYTE = 1.22873
TRAFFIC_SOURCE_SHA = "ec8019b9cf4065de"


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


def derived_fp64_peak_tflops(sms, mhz) -> float:
    """FP64 pipe peak from unit counts and a clock: SMs x 2 DFMA lanes x 2 flops x clock."""
    return sms * DFMA_LANES_PER_SM_CLK * 2 * mhz * 1e6 / 1e12


def kernel_sha() -> str:
    """SHA-256 prefix of the FP64 tile kernels and of the planner that picks their tiles."""
    import hashlib
    h = hashlib.sha256()
    for name in ("fp64_tiles.cu", "api.cu"):
        h.update(open(os.path.join(ROOT, "paper_2311_07602_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def fp64_probe(L, dev_index: int, seconds: float = 2.0) -> dict:
    """The FP64 pipe's throughput measured by lrb_fp64_peak_probe (a DFMA
    kernel over the whole GPU) for about `seconds`, with the SM clock sampled
    while it runs."""
    t_short, ms_short = L.lrb_fp64_peak_probe(dev_index, 1 << 14)
    iters = max(1 << 14, int((1 << 14) * seconds * 1e3 / max(ms_short, 1e-3)))
    s = ClockSampler(dev_index)
    s.start()
    tflops, ms = L.lrb_fp64_peak_probe(dev_index, iters)
    clk = s.stop()
    return {"tflops": tflops, "ms": ms, "iters": iters, "clocks": clk}


# ---- host topology (where pinned host buffers live relative to the GPU) ----

def _cpu_node(cpu: int):
    d = f"/sys/devices/system/cpu/cpu{cpu}"
    try:
        for name in os.listdir(d):
            if name.startswith("node") and name[4:].isdigit():
                return int(name[4:])
    except OSError:
        pass
    return None


def gpu_numa_node(props):
    for dom_fmt in ("{:04x}", "{:08x}"):
        try:
            bdf = (dom_fmt.format(props.pci_domain_id) + f":{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0")
            with open(f"/sys/bus/pci/devices/{bdf}/numa_node") as f:
                return int(f.read().strip())
        except (OSError, ValueError, AttributeError):
            continue
    return None


def page_nodes(ptr: int, nbytes: int, samples: int = 64) -> dict:
    """NUMA nodes of `samples` pages spread over [ptr, ptr + nbytes), from the
    move_pages system call in query mode (nodes = NULL); {} where unsupported."""
    nr = {"aarch64": 239, "x86_64": 279}.get(platform.machine())
    if nr is None or nbytes <= 0:
        return {}
    page = os.sysconf("SC_PAGE_SIZE")
    addrs = [(ptr + (nbytes - 1) * i // max(1, samples - 1)) & ~(page - 1) for i in range(samples)]
    pages = (ctypes.c_void_p * samples)(*addrs)
    status = (ctypes.c_int * samples)()
    libc = ctypes.CDLL(None, use_errno=True)
    libc.syscall.restype = ctypes.c_long
    r = libc.syscall(ctypes.c_long(nr), ctypes.c_int(0), ctypes.c_ulong(samples), pages, None, status, ctypes.c_int(0))
    if r != 0:
        return {"error": os.strerror(ctypes.get_errno())}
    hist = {}
    for v in status:
        hist[str(v)] = hist.get(str(v), 0) + 1
    return hist


def host_topology(props) -> dict:
    cpus = sorted(os.sched_getaffinity(0))
    nodes = {}
    for c in cpus:
        n = _cpu_node(c)
        nodes[str(n)] = nodes.get(str(n), 0) + 1
    return {"allowed_cpus": len(cpus), "cpu_nodes": nodes, "gpu_numa_node": gpu_numa_node(props),
            "host_mem_gb": round(os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 1e9, 1)}


# ---- workloads -------------------------------------------------------------

def variable_workload(device, count=VARIABLE_COUNT, rank=0, world=1, strong=False):
    """The variable-size batch (all of it, or this rank's LPT share)."""
    from paper_2311_07602_gb300 import workloads as W
    forms, bs, rs = W.variable_shapes(VARIABLE_COUNT, seed=3)
    if count != VARIABLE_COUNT:
        forms, bs, rs = forms[:count], bs[:count], rs[:count]
    if strong and world > 1:
        from paper_2311_07602_gb300 import shard
        m = bs.astype(np.int64)
        n = np.where(forms == W.FORM_T, rs, bs).astype(np.int64)
        k = np.where(forms == W.FORM_T, bs, rs).astype(np.int64)
        part = shard.lpt_partition(m, n, k, world)
        sel = np.nonzero(part == rank)[0]
        forms, bs, rs = forms[sel], bs[sel], rs[sel]
    return W.variable_batch(forms, bs, rs, seed=3, device=device, pool_elems=(4 << 30) // 8)


def sweep_batches(device, scale=1.0):
    from paper_2311_07602_gb300 import workloads as W
    return [W.uniform_batch(f, b, r, max(1, int(round(n * scale))), dist="normal", seed=s, device=device)
            for f, b, r, n, s in W.uniform_sweep_groups()]


def variable_sample_cpu(target_flops: float, seed: int = 33):
    """A seeded random sample of the variable-size batch's entries (same
    shapes, same value distribution) whose flops reach `target_flops`, on the
    host (its operand pool is just large enough for the largest operand x 4)."""
    from paper_2311_07602_gb300 import workloads as W
    forms, bs, rs = W.variable_shapes(VARIABLE_COUNT, seed=3)
    m = bs.astype(np.float64)
    n = np.where(forms == W.FORM_T, rs, bs).astype(np.float64)
    k = np.where(forms == W.FORM_T, bs, rs).astype(np.float64)
    f = 2.0 * m * n * k
    order = np.random.default_rng(seed).permutation(VARIABLE_COUNT)
    cnt = int(np.searchsorted(np.cumsum(f[order]), target_flops)) + 1
    sel = np.sort(order[:min(cnt, VARIABLE_COUNT)])
    total_flops = float(f.sum())
    return W.variable_batch(forms[sel], bs[sel], rs[sel], seed=seed, device="cpu"), total_flops


def oracle_run(batch, nthreads: int = 0):
    """The oracle, as it stands, on a host batch: (flops, seconds, threads)."""
    import oracle
    A, B, C = batch.A.numpy(), batch.B.numpy(), batch.C.numpy()
    ents = [dict(A=A, B=B, C=C, offA=int(batch.offA[e]), offB=int(batch.offB[e]), offC=int(batch.offC[e]),
                 m=int(batch.m[e]), n=int(batch.n[e]), k=int(batch.k[e]), lda=int(batch.lda[e]),
                 ldb=int(batch.ldb[e]), ldc=int(batch.ldc[e])) for e in range(len(batch))]
    t0 = time.perf_counter()
    used = oracle.gemm_batch(ents, nthreads=nthreads)
    return batch.flops(), time.perf_counter() - t0, used


def cpu_baseline_variable(target_flops: float = 4e11) -> dict:
    """The oracle on a bounded random sample of the variable-size batch,
    timed on the host cores; also the full batch's time extrapolated by flops."""
    sample, total_flops = variable_sample_cpu(target_flops)
    f, s, used = oracle_run(sample)
    rate = f / s / 1e9
    return {"value": round(rate, 3), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": (f"{len(sample)} of the 20,000 entries drawn at random (seed 33), {f:.3g} flops, {s:.1f} s "
                       f"on the host cores; the full batch ({total_flops:.3g} flops) extrapolates to "
                       f"{total_flops / (rate * 1e9):.0f} s")}


def cpu_baseline_extras() -> dict:
    """The oracle, as it stands, on small samples of the other workloads
    (same shapes and distributions), timed on the host cores: the small
    O-form batch (whole), the uniform sweep (the first 1/32 of every group), the paper's low-rank chain (2000
    blocks, b 1024, r 16; the paper's flop count), the randomized SVD (4
    kernel-matrix blocks, 1024^2, r 16, l 26, q 1; the library's flop count)
    and the split-precision product (4 T-form entries, 1024 x 64 x 1024,
    BF16 S = 3; FP64-equivalent flops)."""
    import oracle
    from oracle import lowrank as OL
    from paper_2311_07602_gb300 import workloads as W
    out = {}
    sm = W.small_o_form(device="cpu")
    ff, ss, used = oracle_run(sm)
    out["small_o_form"] = {"gflops": round(ff / ss / 1e9, 2), "ms": round(ss * 1e3, 2), "threads": used,
                           "sample": "the whole batch (64 x 256x256x16)"}
    fl, secs, ents = 0.0, 0.0, 0
    for f, b, r, n, s in W.uniform_sweep_groups():
        cnt = max(1, n // 32)
        bt = W.uniform_batch(f, b, r, cnt, dist="normal", seed=s, device="cpu")
        ff, ss, used = oracle_run(bt)
        fl += ff
        secs += ss
        ents += cnt
    out["uniform_sweep"] = {"gflops": round(fl / secs / 1e9, 2), "threads": used,
                            "sample": f"first 1/32 of every group ({ents} entries)"}
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
    """The reference arm: the CPU oracle, as it stands, on a bounded random
    sample of the variable-size batch per step (the same sample every step)."""
    rank, _, world = dist_env()
    if world > 1 and rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    sample, total_flops = variable_sample_cpu(args.ref_flops)
    for _ in range(args.warmup):
        oracle_run(sample)
    flops, secs, used = 0.0, 0.0, 1
    for _ in range(args.steps):
        c0 = sample.C.clone()
        f, s, used = oracle_run(sample)
        sample.C.copy_(c0)
        flops += f
        secs += s
    val = flops / secs / 1e9
    desc = (f"{len(sample)} of the 20,000 entries drawn at random (seed 33), {flops / args.steps:.3g} flops per step; "
            f"the full batch ({total_flops:.3g} flops) extrapolates to {total_flops / (val * 1e9):.0f} s")
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": round(val, 3), "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(val, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lrbatch", choices=["lrbatch", "reference"])
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="multi-GPU: every rank runs the whole batch (weak) or its LPT share of it (strong)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--ref-flops", type=float, default=3e10, help="oracle flops per reference-arm step")
    ap.add_argument("--cpu-flops", type=float, default=4e11, help="oracle flops of the cpu_baseline sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads")
    ap.add_argument("--extras", default="sweep,small,split,split_var,serving,dmma,lr,blr,lowrank",
                    help="comma-separated subset of the other workloads (also: sweep_e2e)")
    ap.add_argument("--split-batch", type=int, default=2048, help="entries of the split-precision batch")
    ap.add_argument("--dmma-scale", type=float, default=0.25, help="batch-count scale of the DMMA comparison")
    ap.add_argument("--lr-batch", type=int, default=20000, help="blocks per low-rank chain configuration")
    ap.add_argument("--lr-ranks", default="8,16,32,96,128", help="ranks of the low-rank chain sweep")
    ap.add_argument("--lowrank-count", type=int, default=1024,
                    help="dense blocks of the randomized-SVD / expansion / rounded-addition leg")
    ap.add_argument("--serving-secs", type=float, default=60.0, help="seconds per 0.25-0.9x capacity point")
    ap.add_argument("--overload-secs", type=float, default=10.0, help="seconds per stated overload rate")
    ap.add_argument("--count", type=int, default=VARIABLE_COUNT,
                    help="entries of the headline batch (profiling runs use a small case; the first N of the 20,000)")
    ap.add_argument("--sweep-scale", type=float, default=1.0, help="batch-count scale of the uniform sweep extra")
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
    strong = args.scaling == "strong" and world > 1

    def barrier():
        if pg is not None:
            pg.barrier()

    def max_over_ranks(x: float) -> float:
        if pg is None:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(x: float) -> float:
        if pg is None:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        pg.all_reduce(t)
        return float(t.item())

    from paper_2311_07602_gb300 import lrbatch as L
    cache = os.environ.get("LRB_TUNE_CACHE") or os.path.join(tempfile.gettempdir(), f"lrb_tune_{local_rank}.json")
    os.environ["LRB_TUNE_CACHE"] = cache
    handle = L.Handle(local_rank)
    stream = torch.cuda.Stream(device=dev)
    props = torch.cuda.get_device_properties(dev)

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

    # ---- the headline: the variable-size batch, one persistent graph launch per step
    vb = variable_workload(dev, args.count, rank, world, strong)
    descs = L.descs_for(vb)
    flops = vb.flops()
    alg_bytes = vb.alg_bytes()
    t0 = time.perf_counter()
    plan = handle.plan(descs, use_graph=True)
    plan_s = time.perf_counter() - t0
    info = plan.info()
    probe = fp64_probe(L, local_rank)

    sampler = ClockSampler(local_rank)
    sampler.start()
    total_ms, per = timed(lambda s: plan.launch(s), args.steps, args.warmup)
    clocks = sampler.stop()
    total_ms = max_over_ranks(total_ms)
    all_flops = sum_over_ranks(flops) if strong else world * flops
    value = all_flops * args.steps / (total_ms / 1e3) / 1e9
    ms_per_step = total_ms / args.steps

    run_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    probe_mhz = probe["clocks"].get("sm_mhz") or run_mhz
    peak = probe["tflops"] * run_mhz / probe_mhz
    derived = derived_fp64_peak_tflops(props.multi_processor_count, clocks.get("sm_max_mhz") or 2070.0)
    achieved = flops / (statistics.mean(per) / 1e3) / 1e12
    traffic = None
    if TRAFFIC_PER_ALG_BYTE is not None and kernel_sha() == TRAFFIC_SOURCE_SHA:
        traffic = round(TRAFFIC_PER_ALG_BYTE * alg_bytes)
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "strong" if strong else "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded N(0,1), generated on the device)",
            "config": {"workload": WORKLOAD if args.count == VARIABLE_COUNT else
                       f"{WORKLOAD} (first {args.count} entries)",
                       "entries": int(info["entries"]), "tiles": int(info["items"]), "flops_per_step": flops,
                       "alg_bytes_per_step": alg_bytes, "persistent_grid": int(info["grid"]),
                       "l2": "inputs larger than L2 (%.0f GB per step), no flush" % (alg_bytes / 1e9),
                       "plan_s_incl_tuning": round(plan_s, 2)},
            "gpu_launches": args.steps,
            "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "kernel": "k_persistent (FP64 DFMA tiles)",
                         "peak_source": "measured: lrb_fp64_peak_probe (DFMA kernel, whole GPU) in this run, "
                                        "scaled by the median SM clock of the timed region over the probe's",
                         "probe": {"tflops": round(probe["tflops"], 4), "sm_mhz": probe_mhz, "ms": round(probe["ms"], 1)},
                         "derived_peak": round(derived, 4), "frac_of_derived": round(achieved / derived, 4)},
            "clocks": clocks}

    if not args.no_plain:
        p_ms, _ = timed(lambda s: plan.launch_plain(s), args.plain_steps, 1 + 2)
        p_ms = max_over_ranks(p_ms)
        pval = all_flops * args.plain_steps / (p_ms / 1e3) / 1e9
        line["plain"] = {"value": round(pval, 2), "unit": UNIT, "ms_per_step": round(p_ms / args.plain_steps, 3),
                         "launches_per_step": int(info["groups"])}
        line["vs_plain"] = round(value / pval, 4)
    plan.close()

    if not args.no_e2e:
        line["e2e"] = e2e_leg(L, [vb], args.e2e_steps, args.warmup, barrier, max_over_ranks, world, local_rank,
                              props, strong, sum_over_ranks)
    del vb
    torch.cuda.empty_cache()

    ex = {}
    if not args.no_extras and world == 1:
        ex = extras(L, handle, stream, dev, peak, timed, set(args.extras.split(",")), args, props)
        if not args.no_cpu:
            t0 = time.perf_counter()
            ex["cpu_oracle"] = cpu_baseline_extras()
            ex["cpu_oracle"]["seconds_total"] = round(time.perf_counter() - t0, 1)
        print("extras: " + json.dumps(ex), flush=True)
        line["targets"] = targets_summary(ex)

    if not args.no_cpu and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline_variable(args.cpu_flops)
    handle.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def targets_summary(ex: dict) -> dict:
    """The named targets in a few fields: the split-precision error per preset
    and form (against the FP64 path) with its fraction of the HBM roof, and the
    serving latencies with their sample counts."""
    out = {}
    sp = ex.get("split")
    if sp:
        out["split_rel_err_vs_fp64"] = {f: {k: v["rel_fro_err_vs_fp64"] for k, v in sp[f].items() if k != "fp64"}
                                        for f in ("T", "O") if f in sp}
        out["split_frac_hbm"] = {f: {k: v["frac_hbm"] for k, v in sp[f].items() if k != "fp64"}
                                 for f in ("T", "O") if f in sp}
    sv = ex.get("serving")
    if sv:
        out["serving_p50_p99_ms_n"] = [[p["load"], p["p50_ms"], p["p99_ms"], p["completed"]] for p in sv["points"]]
        out["serving_capacity_req_s"] = sv["capacity_req_s"]
    sw = ex.get("uniform_sweep")
    if sw:
        out["uniform_sweep_gflops"] = sw["gflops"]
        out["uniform_sweep_frac"] = sw["frac_fp64_peak"]
    out["alone_equals_mix"] = "bitwise, tests/test_gpu_serving.py (FP64 and split waves)"
    return out


def extras(L, handle, stream, dev, peak_fp64, timed, which, args, props):
    """The other workloads, each with its own plan."""
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"fp64_peak_tflops": round(peak_fp64, 4)}
    if "sweep" in which:
        out["uniform_sweep"] = sweep_leg(L, handle, dev, peak_fp64, timed, args.sweep_scale)
    if "sweep_e2e" in which:
        bts = sweep_batches(dev, args.sweep_scale)
        out["uniform_sweep_e2e"] = e2e_leg(L, bts, args.e2e_steps, args.warmup, lambda: None, lambda x: x, 1,
                                           dev.index or 0, props, False, lambda x: x)
        del bts
        torch.cuda.empty_cache()
    if "small" in which:
        out["small_o_form"] = small_leg(L, handle, stream, dev, peak_fp64)
    if "split" in which:
        out["split"] = split_leg(L, handle, dev, timed, hbm, args.split_batch)
    if "split_var" in which:
        out["split_variable"] = split_var_leg(L, handle, dev, timed, args.count)
    if "serving" in which:
        out["serving"] = serving_leg(L, handle, dev, peak_fp64, args.serving_secs, args.overload_secs)
    if "dmma" in which:
        out["dmma"] = dmma_leg(L, handle, dev, peak_fp64, timed, args.dmma_scale)
    if "lr" in which:
        out["lr_chain"] = lr_leg(L, handle, dev, peak_fp64, timed, args.lr_batch,
                                 tuple(int(x) for x in args.lr_ranks.split(",")))
    if "blr" in which:
        out["blr_matvec"] = blr_leg(L, handle, dev, peak_fp64, timed)
    if "lowrank" in which:
        out["lowrank"] = lowrank_leg(L, handle, dev, peak_fp64, timed, count=args.lowrank_count)
    return out


def sweep_leg(L, handle, dev, peak_fp64, timed, scale=1.0):
    """The uniform-shape sweep (b in {256, 512, 1024} x r in {16, 32, 64} x
    both forms, 32,256 entries, N(0,1)) as one persistent graph launch,
    through one launch per shape, and every (form, b, r) group as a plan of
    its own."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    batches = sweep_batches(dev, scale)
    descs = np.concatenate([L.descs_for(b) for b in batches])
    f = float(sum(b.flops() for b in batches))
    with handle.plan(descs, use_graph=True) as p:
        info = p.info()
        ms, _ = timed(lambda s: p.launch(s), 5, 3)
        ms_q, _ = timed(lambda s: p.launch_plain(s), 3, 3)
    # every (form, b, r) group on its own: one persistent graph launch each
    groups = []
    for (form, b, r, n, _), bt in zip(W.uniform_sweep_groups(), batches):
        fg = bt.flops()
        with handle.plan(L.descs_for(bt), use_graph=True) as pg:
            ms_g, _ = timed(lambda s: pg.launch(s), 3, 3)
        groups.append({"form": "T" if form == W.FORM_T else "O", "b": b, "r": r, "batch": len(bt),
                       "ms": round(ms_g / 3, 3), "gflops": round(fg * 3 / ms_g / 1e6, 1),
                       "frac_fp64_peak": round(fg * 3 / ms_g / 1e9 / peak_fp64, 4)})
    del batches
    torch.cuda.empty_cache()
    return {"workload": "b in {256,512,1024} (batch 4096/1024/256) x r in {16,32,64} x T/O, N(0,1)"
                        + ("" if scale == 1.0 else f" (batch counts x {scale})"),
            "gflops": round(f * 5 / ms / 1e6, 1), "ms": round(ms / 5, 3),
            "frac_fp64_peak": round(f * 5 / ms / 1e9 / peak_fp64, 4),
            "plain_gflops": round(f * 3 / ms_q / 1e6, 1), "plain_launches": int(info["groups"]),
            "groups": groups}


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


def split_var_leg(L, handle, dev, timed, count=VARIABLE_COUNT):
    """The variable-size batch of the headline in split precision (BF16,
    S = 3): one plan over all entries (pre-passes and both kernel modes in
    one launch), its FP64-equivalent rate, and its error against the FP64
    path from the same C: relative Frobenius norm of the difference of the
    two results over the norm of the FP64 product A B, over the whole batch."""
    import torch
    vb = variable_workload(dev, count)
    f = vb.flops()
    descs = L.descs_for(vb)
    c0 = vb.C.clone()
    out = {"workload": "the headline's variable-size batch (%d entries, N(0,1)), BF16 S = 3" % len(vb)}
    with handle.plan(descs, precision=L.LRB_PREC_SPLIT_BF16_S3) as p:
        info = p.info()
        p.launch()
        torch.cuda.synchronize()
        st = p.status()
        cs = vb.C.clone()
        ms, _ = timed(lambda s: p.launch(s), 3, 3)
    vb.C.copy_(c0)
    with handle.plan(descs, use_graph=True) as p:
        p.launch()
        torch.cuda.synchronize()
    num = den = 0.0
    step = 1 << 27
    for i in range(0, vb.C.numel(), step):
        cf = vb.C[i:i + step]
        num += float(torch.sum((cs[i:i + step] - cf) ** 2))
        den += float(torch.sum((cf - c0[i:i + step]) ** 2))
    out.update({"ms": round(ms / 3, 3), "tflops_fp64_equiv": round(f * 3 / ms / 1e9, 2),
                "items": int(info["items"]), "rel_fro_err_vs_fp64_product": float(f"{(num / den) ** 0.5:.3g}"),
                "status": int(st)})
    del vb, c0, cs
    torch.cuda.empty_cache()
    return out


def split_leg(L, handle, dev, timed, hbm, batch):
    """Split precision (BF16/FP16 x 3/4 digits) against the FP64 path on the
    wide-range batch b 1024, r 64, entries 10^U(-4,4) N(0,1), both forms.  The
    error of each path is measured on one application to a zeroed C against
    the FP64 (DFMA) path's product, whose own error against the oracle the
    tests bound by 1e-13: relative Frobenius error over the whole batch and
    the largest per-entry one.  FP64 DMMA tiles (forced) are measured too."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    res = {}
    paths = (("fp64", dict(precision=L.LRB_PREC_FP64, use_graph=True)),
             ("fp64_dmma", dict(precision=L.LRB_PREC_FP64_DMMA_ALLOWED, use_graph=True, force_variant=9)),
             ("bf16_s3", dict(precision=L.LRB_PREC_SPLIT_BF16_S3)), ("bf16_s4", dict(precision=L.LRB_PREC_SPLIT_BF16_S4)),
             ("fp16_s3", dict(precision=L.LRB_PREC_SPLIT_FP16_S3)), ("fp16_s4", dict(precision=L.LRB_PREC_SPLIT_FP16_S4)))
    for form in (W.FORM_T, W.FORM_O):
        wb = W.wide_range(form, batch=batch, device=dev)
        f = wb.flops()
        ab = wb.alg_bytes()
        m, n = int(wb.m[0]), int(wb.n[0])
        row = {}
        ref = None
        for name, opts in paths:
            with handle.plan(L.descs_for(wb), **opts) as p:
                wb.C.zero_()
                p.launch()
                torch.cuda.synchronize()
                prod = wb.C.view(batch, m * n)
                if ref is None:
                    ref = prod.clone()
                    rnorm = ref.norm(dim=1)
                    err_all, err_max = 0.0, 0.0
                else:
                    d = (prod - ref).norm(dim=1)
                    err_all = float(d.norm() / rnorm.norm())
                    err_max = float((d / rnorm).max())
                steps = 2 if name.startswith("fp64") else 5
                ms, _ = timed(lambda s: p.launch(s), steps, 3)
                st = p.status()
            ms /= steps
            row[name] = {"ms": round(ms, 3), "gflops_fp64_equiv": round(f / ms / 1e6, 1),
                         "hbm_gbs_alg": round(ab / ms / 1e6, 1), "frac_hbm": round(ab / ms / 1e6 / hbm, 4),
                         "rel_fro_err_vs_fp64": float(f"{err_all:.3g}"), "max_entry_rel_err_vs_fp64": float(f"{err_max:.3g}"),
                         "status": int(st)}
        res["T" if form == W.FORM_T else "O"] = row
        del wb, ref
        torch.cuda.empty_cache()
    return {"workload": f"b 1024, r 64, {batch} entries, 10^U(-4,4) N(0,1), seed 4; errors on one application to "
                        f"C = 0 against the FP64 DFMA path", "hbm_peak_gbs": hbm, **res}


def serving_leg(L, handle, dev, peak_fp64, secs=60.0, overload_secs=10.0, budget=40 << 30):
    """Poisson request streams into the continuous-batching queue.  Each
    request: 1..512 products, b log-uniform [64, 2048], r in {8..128}, T/O
    50/50; operands are views into a 4 GB device pool, results go to a 64 GB
    device ring.  Offered loads: 0.25 / 0.5 / 0.75 / 0.9 x the FP64 capacity
    (FP64 peak / mean request flops) for `secs` each, the stated overload rates
    1k / 2k / 5k / 10k / 20k req/s for `overload_secs` each (waiting FIFO
    limited to 32), and 0.9 x the FP64 capacity once more with split-precision
    (BF16, S = 3) waves; 40 GB admission budget, 4 stream slots.  p50/p99 are
    over every completed request of a point (submission -> completion), and
    `completed` is that sample count."""
    import torch
    from paper_2311_07602_gb300 import workloads as W
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    pool = torch.empty((4 << 30) // 8, dtype=torch.float64, device=dev).normal_(generator=g)
    ring = torch.zeros((64 << 30) // 8, dtype=torch.float64, device=dev)
    _, probe = W.serving_requests(2000, 1.0, seed=55)
    mean_flops = float(np.mean([np.sum(2.0 * bb.astype(np.float64) ** 2 * rr) for _, bb, rr in probe]))
    capacity = 0.98 * peak_fp64 * 1e12 / mean_flops
    points = [(f"{fr:g}x capacity", fr * capacity, secs, 4096, L.LRB_PREC_FP64) for fr in (0.25, 0.5, 0.75, 0.9)]
    points += [(f"{r // 1000}k req/s", float(r), overload_secs, 32, L.LRB_PREC_FP64)
               for r in (1000, 2000, 5000, 10000, 20000)]
    points += [("0.9x FP64 capacity, split BF16 S=3 waves", 0.9 * capacity, min(secs, 20.0), 4096,
                L.LRB_PREC_SPLIT_BF16_S3)]
    rng = np.random.default_rng(505)
    cursor = 0
    results = []
    for idx, (label, rate, dur, max_waiting, prec) in enumerate(points):
        count = max(4, int(rate * dur))
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
                        "p99_ms": round(st["p99_ms"], 3), "max_ms": round(st["max_ms"], 3),
                        "sustained_gflops": round(st["gflops"], 1),
                        "waves": int(st["waves"]), "max_concurrent_waves": int(st["max_concurrent_waves"]),
                        "mean_wave_entries": round(st["mean_wave_entries"], 1),
                        "peak_reserved_gb": round(st["peak_reserved_bytes"] / 1e9, 2)})
    del pool, ring
    torch.cuda.empty_cache()
    return {"workload": "Poisson requests, 1..512 products each, b log-uniform [64,2048], r in {8..128}, "
                        "T/O 50/50, N(0,1), FP64, 40 GB budget, 4 stream slots",
            "mean_request_gflop": round(mean_flops / 1e9, 2), "capacity_req_s": round(capacity, 1),
            "points": results}


def e2e_leg(L, batches, steps, warmup, barrier, max_over_ranks, world, dev_index, props, strong, sum_over_ranks):
    """The same work through lrb_execute_host: the operands in pinned host
    memory, their host->device copies, the launches and the device->host copy
    of every C in the timed region (the call returns after host C holds the
    result).  With N ranks in weak scaling every rank takes the first 1/N of
    each batch's entries (host memory is shared by the ranks); flops count
    what ran.  Also reported: the per-engine breakdown of the last call
    (lrb_execute_host_get_timing), the pinned-copy rates of a single large
    copy each way from a fresh pinned buffer and from the caller's own
    buffers, and where the pinned pages live relative to the GPU."""
    import torch
    handle = L.Handle(dev_index)
    rows, hold = [], []
    h2d = d2h = 0
    fl = 0.0
    topo = host_topology(props)
    pages = {}
    for bi, b in enumerate(batches):
        cnt = len(b) if (world == 1 or strong) else max(1, len(b) // world)
        sel = np.arange(cnt)
        host = {}
        ends = {}
        for key, off, ld, cols in (("A", b.offA, b.lda, b.k), ("B", b.offB, b.ldb, b.n), ("C", b.offC, b.ldc, b.n)):
            t = getattr(b, key)
            end = int(np.max(off[sel] + ld[sel].astype(np.int64) * cols[sel]))
            ends[t.data_ptr()] = max(ends.get(t.data_ptr(), 0), end)
        for key in ("A", "B", "C"):
            t = getattr(b, key)
            if t.data_ptr() in host:
                continue
            n_el = ends[t.data_ptr()]
            hb = torch.empty(n_el, dtype=torch.float64, pin_memory=True)
            hb.copy_(t[:n_el])
            host[t.data_ptr()] = hb
            hold.append(hb)
            if bi == 0:
                pages[key] = page_nodes(hb.data_ptr(), 8 * n_el)
        hA, hB, hC = (host[getattr(b, key).data_ptr()] for key in ("A", "B", "C"))
        d = np.zeros(cnt, dtype=L.DESC_DTYPE)
        d["A"] = np.uint64(hA.data_ptr()) + 8 * b.offA[sel].astype(np.uint64)
        d["B"] = np.uint64(hB.data_ptr()) + 8 * b.offB[sel].astype(np.uint64)
        d["C"] = np.uint64(hC.data_ptr()) + 8 * b.offC[sel].astype(np.uint64)
        for key in ("m", "n", "k", "lda", "ldb", "ldc"):
            d[key] = getattr(b, key)[sel]
        rows.append(d)
        m, n, k = (getattr(b, key)[sel].astype(np.float64) for key in ("m", "n", "k"))
        fl += float(np.sum(2.0 * m * n * k))
    descs = np.concatenate(rows)
    # the box's pinned-copy rates in this run (context for the e2e figure):
    # the largest pinned buffer (up to 4 GB) in, then out, then both at once
    nel = (4 << 30) // 8
    src = torch.zeros(nel, dtype=torch.float64, pin_memory=True)
    dbuf = torch.zeros(nel, dtype=torch.float64, device="cuda")
    dbuf2 = torch.zeros(nel, dtype=torch.float64, device="cuda")
    copy_gbs = {}
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    for name in ("h2d", "d2h", "both"):
        for rep in range(2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s_in.wait_event(e0)
            s_out.wait_event(e0)
            if name in ("h2d", "both"):
                with torch.cuda.stream(s_in):
                    dbuf.copy_(src, non_blocking=True)
            if name in ("d2h", "both"):
                with torch.cuda.stream(s_out):
                    src.copy_(dbuf2, non_blocking=True)
            torch.cuda.current_stream().wait_stream(s_in)
            torch.cuda.current_stream().wait_stream(s_out)
            e1.record()
            torch.cuda.synchronize()
        copy_gbs[name] = round((2 if name == "both" else 1) * 8 * nel / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    del dbuf, dbuf2, src
    torch.cuda.synchronize()
    handle.set_host_timing(True)
    stream = torch.cuda.Stream()
    for _ in range(warmup):
        handle.execute_host(descs, stream)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        handle.execute_host(descs, stream)
    torch.cuda.synchronize()
    barrier()
    secs = max_over_ranks(time.perf_counter() - t0)
    tm = handle.host_timing()
    handle.close()
    # the same single large copies from and into the caller's own pinned
    # buffers (the operand pool in, the start of C out), after the timed
    # region: a fresh pinned buffer can copy at full rate while these do not
    torch.cuda.synchronize()
    own_gbs = {}
    for name, hb, to_dev in (("pool_h2d", hA, True), ("C_d2h", hC, False)):
        n_el = min(hb.numel(), (4 << 30) // 8)
        dbuf = torch.empty(n_el, dtype=torch.float64, device="cuda")
        best = 0.0
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if to_dev:
                dbuf.copy_(hb[:n_el], non_blocking=True)
            else:
                hb[:n_el].copy_(dbuf, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, 8 * n_el / (e0.elapsed_time(e1) / 1e3) / 1e9)
        own_gbs[name] = round(best, 1)
        del dbuf
    h2d = int(tm["h2d_bytes"])
    d2h = int(tm["d2h_bytes"])
    all_fl = sum_over_ranks(fl) if strong else world * fl
    del hold
    if hasattr(torch._C, "_host_emptyCache"):
        torch._C._host_emptyCache()          # hand the pinned buffers back before the next leg
    return {"value": round(all_fl * steps / secs / 1e9, 2), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "flops_per_step_per_rank": fl,
            "last_call": {"wall_ms": round(tm["wall_ms"], 1), "pieces": int(tm["pieces"]),
                          "h2d_busy_ms": round(tm["h2d_busy_ms"], 1), "compute_busy_ms": round(tm["compute_busy_ms"], 1),
                          "d2h_busy_ms": round(tm["d2h_busy_ms"], 1),
                          "h2d_gbs": round(tm["h2d_bytes"] / max(tm["h2d_busy_ms"], 1e-9) / 1e6, 1),
                          "d2h_gbs": round(tm["d2h_bytes"] / max(tm["d2h_busy_ms"], 1e-9) / 1e6, 1),
                          "overlap_h2d_compute_ms": round(tm["overlap_h2d_compute_ms"], 1),
                          "overlap_d2h_compute_ms": round(tm["overlap_d2h_compute_ms"], 1),
                          "overlap_h2d_d2h_ms": round(tm["overlap_h2d_d2h_ms"], 1),
                          "first_launch_after_ms": round(tm["compute_start_ms"], 1),
                          "copies_after_last_launch_ms": round(tm["compute_end_to_last_ms"], 1),
                          "first_piece_h2d_ms": round(tm["first_h2d_ms"], 1),
                          "first_piece_h2d_gb": round(tm["first_h2d_bytes"] / 1e9, 3)},
            "pinned_copy_gbs": copy_gbs, "caller_buffer_copy_gbs": own_gbs, "host": topo, "pinned_page_nodes": pages,
            "api": "lrb_execute_host (pinned host buffers; copies in, compute and copies out pipelined in pieces)"}


if __name__ == "__main__":
    sys.exit(main())
