#!/usr/bin/env python
"""Benchmark of the reverse k-MIPS top-N hot path on one GB300 (or N replicas).

One step = one rkm_topn call on the largest single-GPU workload, MF-like users
n=2,000,000, items m=500,000, d=128, k=10, N=100 (FP32 grid inputs, resident in HBM):
prep, thresholds (product + selector + exact rescoring), Eq. 2 bounds, filtered counting,
band rescoring, top-N.  After the timed BF16 steps the same inputs run once through the
FP8 and the plain exact FP32 paths; their top-N, tau_u and t_u must equal the BF16 path's
bit for bit (the run fails otherwise) and the step-time ratios are reported.

metric: user-item pairs scored per second = n*m / step time (the dense pair count of
the problem, whatever the filter skips).  L2 is flushed (a 512 MiB write) before each
timed step, outside the timed events.

--impl reference times the FP64 oracle on the host cores on a bounded user sample of
the same workload (the CPU baseline; the paper has no GPU implementation).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "user-item pairs scored/sec (end-to-end top-N)"
UNIT = "pairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp8", "fp32"])
    ap.add_argument("--workload", default="mf-2m-k10")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--n", type=int, default=None, help="override the number of users (profiling cases)")
    ap.add_argument("--m", type=int, default=None, help="override the number of items (profiling cases)")
    ap.add_argument("--scores", default="count", choices=["count", "histogram"],
                    help="rkm_topn scores: counting pass with the Eq. 2 filter (default, every step of the"
                         " path), or the histogram of the exact S_k(u) lists of the threshold pass")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP8 and FP32 runs on the same inputs (identical results, speedups)")
    ap.add_argument("--epilogue-groups", type=int, default=0, choices=[0, 2, 4],
                    help="warpgroups reading each accumulator tile in the tensor-core kernels (0 = auto)")
    ap.add_argument("--no-seed-order", action="store_true",
                    help="tensor-core threshold pass with users in input order (no seed pass)")
    ap.add_argument("--requests", type=int, default=2000, help="serve-1m: requests per offered load")
    ap.add_argument("--slots", type=int, default=2, help="serve-1m: concurrent batches of the serving loop")
    return ap.parse_args()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.reader = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        p["source"] = "measured"
        return p
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


# DRAM bytes per launch of the threshold kernel from an ncu capture (read + write, taken on a
# 131,072-user call of the same items and scaled by the users processed to the benchmark
# call; with the seed order a call makes two launches, the seed pass and the main pass, and
# the figure is their mean, like the kernel time of the roofline), keyed by a hash of the
# kernel sources: when the kernel changes, the counters no longer apply (None).
THRESHOLD_TRAFFIC = {
    "c05a61984b4add74abe8133b08ca34888d55899a2c766065e30a230ff1e3fbf4": {"mf-2m-k10": 5.05e+09, "mf-500k": 5.72e+08},
}
KERNEL_SOURCES = ['tc.cu', 'epilogue.cuh', 'tc_ptx.cuh', 'common.cuh']


def threshold_traffic(workload: str):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2504_13445_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return THRESHOLD_TRAFFIC.get(h.hexdigest(), {}).get(workload)


def tensor_peak(peaks: dict, precision: str, sustained: bool = False):
    """Dense tensor peak of the product's dtype: the measured BF16 figure (burst for a kernel
    timed alone, sustained for one timed inside a seconds-long run of steps), times the
    nominal FP8/BF16 ratio (4.5 / 2.25 PFLOP/s) for FP8."""
    key = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in peaks else "bf16_tflops"
    kind = "sustained" if key.endswith("sustained") else "burst"
    bf16 = peaks[key]
    if precision == "fp8":
        return 2.0 * bf16, f"{peaks['source']} {key} ({kind}) x 2 (nominal FP8/BF16 dense ratio)"
    return bf16, f"{peaks['source']} {key} ({kind})"


DTYPE = {"bf16": "bf16", "fp8": "e4m3", "fp32": "f32"}


def fp32_alu_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    # 128 FP32 FMA lanes per SM, 2 FLOP per FMA.
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def cpu_baseline(W, workload: str, seconds: float, n=None, m=None) -> dict:
    """The oracle as it stands on the host cores, on users [0, S) of the workload against
    every item (Definition 1 thresholds and the histogram of S_k(u)), S grown in blocks
    until about `seconds` of work.  Runs in a spawned child so BLAS threads are pinned."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_cpu_child, args=(workload, W.k, seconds, q, n, m))
    p.start()
    res = q.get()
    p.join()
    return res


def _cpu_child(cfg, k, seconds, q, n=None, m=None):
    threads = os.cpu_count() or 1
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["MKL_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    import numpy as np  # noqa: F401
    import oracle
    import workloads
    over = {key: v for key, v in (("n", n), ("m", m)) if v}
    n_all = dict(workloads.CONFIGS[cfg], **over)["n"]
    P = workloads.rows(cfg, "P", **over)
    block = 64 * threads
    done, dt = 0, 0.0
    while True:
        Ub = workloads.rows(cfg, "U", done, block, **over)  # drawn outside the timed work
        t0 = time.perf_counter()
        tau, tid, topk = oracle.kmips(Ub, P, k, block=64, threads=threads)
        oracle.scores_histogram(topk, P.shape[0])
        dt += time.perf_counter() - t0
        done += Ub.shape[0]
        if dt >= seconds or done >= n_all:
            break
    q.put({"value": done * P.shape[0] / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"users [0,{done}) x all {P.shape[0]} items of {cfg}: FP64 thresholds + histogram, {dt:.1f} s"})


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores: each step is a bounded user sample."""
    if rank != 0:
        return
    if args.workload == "serve-1m":
        return run_reference_serve(args)
    if args.workload == "batch-64":
        return run_reference_batch(args)
    import oracle
    import workloads
    threads = os.cpu_count() or 1
    over = {key: v for key, v in (("n", args.n), ("m", args.m)) if v}
    cfg = dict(workloads.CONFIGS[args.workload], **over)
    P = workloads.rows(args.workload, "P", **over)
    # The same blocking as the cpu_baseline leg: 64 users per oracle block, one block per
    # host thread per step; each step's users are drawn before its timer starts.
    sample = min(64 * threads, cfg["n"])
    times = []
    for step in range(args.warmup + args.steps):
        u0 = (step * sample) % max(1, cfg["n"] - sample + 1)
        Ub = workloads.rows(args.workload, "U", u0, sample, **over)
        t0 = time.perf_counter()
        tau, tid, topk = oracle.kmips(Ub, P, cfg["k"], block=64, threads=threads)
        oracle.scores_histogram(topk, P.shape[0])
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    ms = 1000 * statistics.mean(times)
    m = P.shape[0]
    value = sample * m / (ms / 1000)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": cfg["n"], "m": m, "d": cfg["d"], "k": cfg["k"],
                       "N": cfg["N"], "sample_users_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} users x all {m} items per step (FP64 thresholds + histogram)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)



def _reference_line(args, value, ms, config, sample, dtype="f64", metric=METRIC):
    threads = os.cpu_count() or 1
    return {"impl": "reference", "metric": metric, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_batch(args):
    """Oracle on the 64-instance batch: each step scores a user sample of one instance (in turn)
    against all of its items; value = sampled pairs / time."""
    import oracle
    import workloads
    threads = os.cpu_count() or 1
    sizes = workloads.batching_instances(64)
    sample = 16 * threads
    times, pairs = [], []
    for step in range(args.warmup + args.steps):
        sz = sizes[step % len(sizes)]
        W = workloads.mf(min(sz["n"], sample), sz["m"], sz["d"], sz["k"], sz["N"], seed=sz["seed"])
        t0 = time.perf_counter()
        tau, tid, topk = oracle.kmips(W.U, W.P, W.k, block=16, threads=threads)
        oracle.scores_histogram(topk, W.m)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            pairs.append(W.n * W.m)
    value = sum(pairs) / sum(times)
    print(json.dumps(_reference_line(
        args, value, 1000 * statistics.mean(times),
        {"workload": "batch-64", "instances": len(sizes), "sample_users_per_step": sample},
        f"users [0,{sample}) of one instance per step x all its items (FP64 thresholds + histogram)")), flush=True)


def run_reference_serve(args):
    """Oracle on the serving workload: thresholds of a user sample against the whole
    catalogue (not timed), then each step scores one request's candidates against the sample
    (Definition 2 for new items); value = sampled user-candidate pairs / time."""
    import oracle
    import workloads
    S = workloads.SERVING
    threads = os.cpu_count() or 1
    sample = 8 * threads
    W = workloads.mf(sample, S["m"], S["d"], S["k"], 1, seed=S["catalog_seed"])
    tau, tid, _ = oracle.kmips(W.U, W.P, W.k, block=8, threads=threads)
    R = args.warmup + args.steps
    _, sizes, offsets = workloads.serving_stream(R, 1.0, seed=S["query_seed"])
    Q = workloads.queries(int(sizes.sum()), W.d, seed=S["query_seed"])
    times, pairs = [], []
    for j in range(R):
        t0 = time.perf_counter()
        oracle.query_new_items(W.U, tau, Q[offsets[j]:offsets[j] + sizes[j]])
        dt = time.perf_counter() - t0
        if j >= args.warmup:
            times.append(dt)
            pairs.append(sample * int(sizes[j]))
    value = sum(pairs) / sum(times)
    print(json.dumps(_reference_line(
        args, value, 1000 * statistics.mean(times),
        {"workload": "serve-1m", "sample_users": sample, "requests": args.steps},
        f"{sample} resident users (thresholds vs all {S['m']} items) x one request per step",
        metric="user-item pairs scored/sec (serving what-if queries)")), flush=True)

def workload(args):
    import workloads
    over = {}
    if args.n:
        over["n"] = args.n
    if args.m:
        over["m"] = args.m
    return workloads.make(args.workload, **over)


def run_ours(args, rank, local, world):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_13445_gb300 as rkm
    import workloads

    torch.cuda.set_device(local)
    W = workload(args)
    U = torch.from_numpy(W.U).cuda()
    P = torch.from_numpy(W.P).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ctx = rkm.Context(args.precision, device=local, profile=True, scores_from_topk=args.scores == "histogram",
                      epilogue_groups=args.epilogue_groups, seed_order=not args.no_seed_order)
    # The result every other path must reproduce bit for bit (top-N, tau_u, t_u).
    ref_out = [x.cpu() for x in ctx.topn(U, P, W.k, W.N, return_thresholds=True)]
    for _ in range(args.warmup):
        ctx.topn(U, P, W.k, W.N)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    torch.cuda.synchronize()
    step_ms, thr_ms, thr_launch, launches, counted, cand, band, evald, thr_pairs = [], [], [], 0, [], [], [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ids, tops = ctx.topn(U, P, W.k, W.N)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = ctx.stats()
        thr_ms.append(st["phase_ms"]["threshold"])
        thr_launch.append(st["threshold_launches"])
        launches += st["kernel_launches"]
        counted.append(st["items_counted"])
        cand.append(st["candidates"])
        band.append(st["band_pairs"])
        evald.append(st["pairs_evaluated"])
        thr_pairs.append(st["threshold_pairs"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    total_ms = max_over_ranks(sum(step_ms), world)
    ms = total_ms / args.steps
    pairs = W.n * W.m
    value = world * pairs / (ms / 1000)

    # End to end through the host-buffer entry point: pinned host inputs, copies inside.
    e2e = None
    if not args.no_e2e:
        Uh = torch.from_numpy(W.U).pin_memory()
        Ph = torch.from_numpy(W.P).pin_memory()
        Un, Pn = Uh.numpy(), Ph.numpy()
        ctx.topn_host(Un, Pn, W.k, W.N)
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(3, args.steps // 2)):
            t0 = time.perf_counter()
            ctx.topn_host(Un, Pn, W.k, W.N)
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.mean(ts), world)
        e2e = {"value": world * pairs / e2e_s, "unit": UNIT, "ms_per_step": 1000 * e2e_s,
               "h2d_bytes_per_step": int(W.U.nbytes + W.P.nbytes), "d2h_bytes_per_step": int(8 * W.N),
               "api": "rkm_topn_host", "phase_ms_last_step": ctx.stats()["phase_ms"]}
    ctx.close()

    # The same inputs through the other precision paths: identical integer results (asserted)
    # and the step-time ratios (the guarded paths against the plain exact FP32 path).
    compare = None
    if not args.no_compare:
        compare = compare_paths(args, rkm, U, P, W, ref_out, local, statistics.mean(step_ms), flush)

    if rank != 0:
        return
    peaks = measured_peaks()
    # Thresholds of very many users may run as several launches (user slices whose candidate
    # lists fit the memory budget): per launch, the users of one slice.
    launches_per_call = statistics.mean(thr_launch)
    thr_avg = statistics.mean(t / max(1, l) for t, l in zip(thr_ms, thr_launch))
    # Algorithmic work of the threshold kernel: 2d FLOP per user-item product it computed
    # (the dense n*m less the item tiles its Cauchy-Schwarz stop skipped).
    flops = 2.0 * statistics.mean(thr_pairs) * W.d / max(1.0, launches_per_call)
    achieved = flops / (thr_avg / 1000) / 1e12
    if args.precision in ("bf16", "fp8"):
        # The steps run back to back for seconds, so the kernel is timed inside a long run:
        # the sustained peak is the denominator; the burst fraction is reported beside it.
        peak, src = tensor_peak(peaks, args.precision, sustained=True)
        burst, _ = tensor_peak(peaks, args.precision)
        roof = {"bound": "tensor", "kernel": "k_threshold_tc (threshold product + selector)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": threshold_traffic(args.workload) if not (args.n or args.m) and args.precision == "bf16"
                else None,
                "peak_source": src, "frac_of_burst": achieved / burst, "burst_peak": burst}
    else:
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = fp32_alu_peak_tflops(sm_mhz)
        roof = {"bound": "alu", "kernel": "k_threshold_simt (threshold product + selector)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": f"152 SMs x 128 FP32 FMA/clk x 2 x {sm_mhz:.0f} MHz"}
    roof["kernel_ms"] = thr_avg
    roof["algorithmic_flops_per_launch"] = flops
    roof["launches_per_step"] = launches_per_call
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload if not (args.n or args.m) else f"{args.workload} resized",
                       "n": W.n, "m": W.m, "d": W.d, "k": W.k, "N": W.N,
                       "precision": args.precision, "inputs": "FP32 on the 2^-12 grid, MF-like",
                       "scores": "counting pass + Eq. 2 filter" if args.scores == "count"
                                 else "histogram of the exact S_k(u) lists (no counting pass)",
                       "l2": "flushed (512 MiB write) before each timed step",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "gpu_launches": int(launches),
            "clocks": clk,
            "detail": {"band_hit_fraction": (statistics.mean(band) /
                                             max(1.0, statistics.mean(evald) - statistics.mean(thr_pairs))
                                             if args.scores == "count" else None),
                       "band_hit_fraction_of": "counting-pass pairs (evaluated pairs minus the threshold pass's)",
                       "threshold_pairs_fraction": statistics.mean(thr_pairs) / (W.n * W.m),
                       "candidates_per_user": statistics.mean(cand) / W.n,
                       "items_counted_mean": statistics.mean(counted), "candidates_mean": statistics.mean(cand),
                       "band_pairs_mean": statistics.mean(band), "pairs_evaluated_mean": statistics.mean(evald),
                       "retries_last_step": st["retries"], "phase_ms_last_step": st["phase_ms"]}}
    if e2e:
        line["e2e"] = e2e
    if compare:
        line["detail"]["paths"] = compare
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(W, args.workload, args.cpu_seconds, args.n, args.m)
    print(json.dumps(line), flush=True)


def compare_paths(args, rkm, U, P, W, ref_out, local, main_ms, flush):
    """Run the workload through every other precision path: one untimed call (workspace
    growth), one timed call.  Each result must equal the main path's top-N ids and scores,
    tau_u and t_u exactly; a mismatch stops the benchmark."""
    import torch
    out = {args.precision: {"ms_per_step": main_ms}}
    stream = torch.cuda.current_stream()
    for prec in ("bf16", "fp8", "fp32"):
        if prec == args.precision:
            continue
        with rkm.Context(prec, device=local, profile=True, scores_from_topk=args.scores == "histogram",
                         epilogue_groups=args.epilogue_groups, seed_order=not args.no_seed_order) as c:
            c.topn(U, P, W.k, W.N)
            torch.cuda.synchronize()
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = c.topn(U, P, W.k, W.N, return_thresholds=True)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            st = c.stats()
        res = [x.cpu() for x in res]
        names = ("top-N ids", "top-N scores", "tau", "tid")
        for name, a, b in zip(names, res, ref_out):
            if not torch.equal(a, b):
                raise SystemExit(f"bench: the {prec} path's {name} differ from the {args.precision} path's")
        counting = st["pairs_evaluated"] - st["threshold_pairs"]
        out[prec] = {"ms_per_step": ms, "identical_results": True,
                     "phase_ms": st["phase_ms"], "candidates_per_user": st["candidates"] / W.n,
                     "band_hit_fraction": st["band_pairs"] / max(1, counting) if args.scores == "count" else None,
                     "band_pairs": st["band_pairs"], "counting_pairs": counting,
                     "threshold_pairs": st["threshold_pairs"], "retries": st["retries"]}
    if "fp32" in out and args.precision != "fp32":
        out["speedup_vs_fp32"] = {p: out["fp32"]["ms_per_step"] / v["ms_per_step"]
                                  for p, v in out.items() if p in ("bf16", "fp8")}
    return out


def run_batch(args, rank, local, world):
    """The 64-instance batch (users log-uniform in [1e4, 1e6], items in [5e3, 2e5], d in
    {32, 64, 128}, k in {5, 10, 25}, N = 20): one rkm_topn_batch per step, BF16, autotuned
    counting tiles, graph replayed after the first call."""
    import tempfile

    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_13445_gb300 as rkm
    import workloads

    torch.cuda.set_device(local)
    sizes = workloads.batching_instances(64)
    if args.n:  # shrink every instance (smoke runs)
        sizes = [dict(sz, n=max(64, sz["n"] // args.n), m=max(64, sz["m"] // args.n)) for sz in sizes]
    probs = []
    for sz in sizes:
        W = workloads.mf(sz["n"], sz["m"], sz["d"], sz["k"], sz["N"], seed=sz["seed"])
        probs.append((torch.from_numpy(W.U).cuda(), torch.from_numpy(W.P).cuda(), W.k, W.N))
    pairs = sum(sz["n"] * sz["m"] for sz in sizes)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    cache = os.path.join(tempfile.gettempdir(), "rkm_tune_cache.txt")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = rkm.Context(args.precision, device=local, autotune=True, tune_cache=cache)
        outs = None
        for _ in range(args.warmup):
            outs = ctx.topn_batch(probs, outs)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        barrier(world)
        clocks.start()
        step_ms, launches = [], 0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = ctx.topn_batch(probs, outs)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            launches += ctx.stats()["kernel_launches"]
        clk = clocks.stop()
        barrier(world)
    ms = max_over_ranks(sum(step_ms), world) / args.steps
    if rank != 0:
        return
    line = {"metric": METRIC, "value": world * pairs / (ms / 1000), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": {"workload": "batch-64", "instances": len(sizes), "pairs": pairs,
                       "users": sum(sz["n"] for sz in sizes), "items": sum(sz["m"] for sz in sizes),
                       "precision": args.precision, "graph": "captured on the first call, replayed",
                       "autotune": "counting work-unit size and first-stage size per size bucket",
                       "l2": "flushed (512 MiB write) before each timed step"},
            "roofline": None, "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


def run_serve(args, rank, local, world):
    """Serving: 1,000,000 resident users (d=100) with thresholds at k=20 against a
    300,000-item catalogue (computed on the device by rkm_thresholds before timing), then
    streams of what-if requests (log-uniform sizes in [1, 4096], candidates from the item
    generator) through the serving loop with host buffers.  First every request is queued at
    once (saturation: the largest throughput the loop sustains), then Poisson arrivals at 25,
    50 and 90% of that throughput, each reporting p50/p99 latency (submit -> counts in the
    caller's buffer).  value = resident users x candidates scored / s at saturation."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_13445_gb300 as rkm
    import workloads

    torch.cuda.set_device(local)
    S = dict(workloads.SERVING)
    if args.n:
        S["n"] = args.n
    if args.m:
        S["m"] = args.m
    W = workloads.mf(S["n"], S["m"], S["d"], S["k"], 1, seed=S["catalog_seed"])
    U = torch.from_numpy(W.U).cuda()
    P = torch.from_numpy(W.P).cuda()
    ctx = rkm.Context(args.precision, device=local, profile=True)
    tau, tid, _ = ctx.thresholds(U, P, W.k)
    ctx.resident_set(U, tau, tid)
    del P
    R = args.requests
    gaps, sizes, offsets = workloads.serving_stream(R, 1.0, seed=S["query_seed"])
    Qall = workloads.queries(int(sizes.sum()), W.d, seed=S["query_seed"])
    reqs = [Qall[o:o + q] for o, q in zip(offsets, sizes)]
    items_total = int(sizes.sum())
    mean_q = float(sizes.mean())

    srv = rkm.Server(ctx, slots=args.slots, max_batch_items=8192, memory_bytes=256 << 20)

    def run_stream(arrivals):
        srv.reset_stats()
        tickets = [None] * R
        t0 = time.perf_counter()
        for j in range(R):
            if arrivals is not None:
                delay = arrivals[j] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            tickets[j] = srv.submit(reqs[j])
        for t in tickets:
            srv.wait(t)
        return srv.stats()

    for _ in range(max(1, args.warmup)):
        run_stream(None)
    clocks = ClockSampler(local)
    clocks.start()
    sat = run_stream(None)
    clk = clocks.stop()
    loads = []
    for frac in (0.25, 0.5, 0.9):
        rate = frac * sat["items_per_s"] / mean_q  # requests per second
        st = run_stream(gaps / rate)
        loads.append({"offered_frac_of_saturation": frac, "rate_req_per_s": rate, "p50_ms": st["p50_ms"],
                      "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
                      "items_per_s": st["items_per_s"], "mean_batch_items": st["mean_batch_items"],
                      "max_in_flight": st["max_in_flight"]})
    srv.close()

    # The dominant kernel (the counting product of one full batch of 8192 candidates), timed
    # alone with CUDA events around each phase.
    Qb = torch.from_numpy(np.ascontiguousarray(Qall[:8192])).cuda()
    ctx.query_new_items(Qb)
    cms = []
    for _ in range(5):
        ctx.query_new_items(Qb)
        cms.append(ctx.stats()["phase_ms"]["count"])
    qst = ctx.stats()
    count_ms = statistics.median(cms)
    flops = 2.0 * qst["pairs_evaluated"] * W.d
    achieved = flops / (count_ms / 1000) / 1e12
    peaks = measured_peaks()
    tc = args.precision in ("bf16", "fp8")
    if tc:
        peak, src = tensor_peak(peaks, args.precision)
    else:
        peak, src = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0)), "FP32 ALU"
    roof = {"bound": "tensor" if tc else "alu",
            "kernel": "k_count_tc (counting product + classify)" if tc else "k_count_simt (counting product + classify)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "peak_source": src,
            "kernel_ms": count_ms, "algorithmic_flops_per_launch": flops,
            "units": "2 d FLOP per evaluated (user, candidate) pair, 8192 candidates"}
    if rank != 0:
        return
    value = world * sat["pairs_per_s"]
    req_bytes = mean_q * W.d * 4
    line = {"metric": "user-item pairs scored/sec (serving what-if queries)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": R, "warmup": max(1, args.warmup),
            "ms_per_step": sat["window_ms"] / R, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": "serve-1m", "users": W.n, "catalogue": W.m, "d": W.d, "k": W.k,
                       "requests": R, "candidates": items_total, "sizes": "log-uniform [1, 4096]",
                       "slots": args.slots, "max_batch_items": 8192, "arena_bytes": 256 << 20,
                       "step": "one request",
                       "l2": "not flushed: the resident users (1M x 128 BF16 = 256 MB) exceed L2, so every"
                             " batch streams them from HBM"},
            "serving": {"saturation": {k: sat[k] for k in ("items_per_s", "p50_ms", "p99_ms", "mean_batch_items",
                                                            "batches", "max_in_flight", "window_ms")},
                        "loads": loads},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(req_bytes),
                    "d2h_bytes_per_step": int(mean_q * 4),
                    "api": "rkm_serve_submit/rkm_serve_wait with host buffers (value is end to end)"},
            "roofline": roof, "gpu_launches": int(sat["kernel_launches"]), "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, local, world = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch-64":
        run_batch(args, rank, local, world)
    elif args.workload == "serve-1m":
        run_serve(args, rank, local, world)
    else:
        run_ours(args, rank, local, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
