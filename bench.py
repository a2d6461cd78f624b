#!/usr/bin/env python
"""Benchmark: time-to-dendrogram and effective pair-distance rate of exact NNM single
linkage on one GB300, through the C ABI.

A step is one pass of the whole path on resident synthetic data: nnm_create (checks,
centring, operand layout), nnm_cluster (all-pairs candidate sweep, exact binary64
re-rank, merge rounds, edge sort, restriction walk, labels) and nnm_destroy.
value = N(N-1)/2 / time-to-dendrogram, in G pair-distances/s (all ranks summed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp16|fp32]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G pair-distances/s and time-to-dendrogram at N=2M,d=25 (BF16+FP64-rerank vs FP32)"
UNIT = "Gpairs/s"
DEFAULT_WORKLOAD = "nnm_n2097152_d25"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="bf16x3", choices=["bf16", "bf16x3", "fp16", "fp32"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--n", type=int, default=None, help="override N (smaller runs)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-peaks", action="store_true", help="skip the FP32/FP64 peak microbenchmarks")
    p.add_argument("--compare", default="fp16,bf16,fp32", help="comma list of other precisions timed for one step each (after one untimed step)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--ref-seconds", type=float, default=None, help="oracle seconds per step of --impl reference")
    return p.parse_args()


# ------------------------------------------------------------------------------------
# distributed plumbing: replicas only (the method's partition is not sharded here)
# ------------------------------------------------------------------------------------

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# ------------------------------------------------------------------------------------

def oracle_pair_rate(X, seconds, seed=0):
    """Exact binary64 1-NN of sampled rows against all rows with the oracle, every core.
    Returns (Gpairs/s, rows sampled, seconds, cores)."""
    import oracle
    oracle.build()
    N = X.shape[0]
    rng = np.random.default_rng(seed)
    rows = rng.choice(N, size=min(16, N), replace=False)
    t0 = time.perf_counter()
    oracle.knn(X, 1, queries=rows)
    t1 = time.perf_counter() - t0
    R = int(min(max(16, 16 * seconds / max(t1, 1e-3)), N))
    rows = rng.choice(N, size=R, replace=False)
    t0 = time.perf_counter()
    oracle.knn(X, 1, queries=rows)
    dt = time.perf_counter() - t0
    return R * (N - 1) / dt / 1e9, R, dt, os.cpu_count()


def run_reference(args, world, rank):
    from paper_1402_3789_gb300.inputs import make
    if rank != 0:
        return
    X = make(args.workload, n=args.n)
    N, d = X.shape
    per_step = args.ref_seconds if args.ref_seconds else max(2.0, min(20.0, 150.0 / max(args.steps + args.warmup, 1)))
    rates = []
    for s in range(args.warmup + args.steps):
        rate, R, dt, cores = oracle_pair_rate(X, per_step, seed=s)
        if s >= args.warmup:
            rates.append((rate, R, dt))
    value = statistics.median(r for r, _, _ in rates)
    R = rates[-1][1]
    ms = statistics.mean(dt for _, _, dt in rates) * 1e3
    sample = (f"exact binary64 1-NN of {R} sampled rows against all {N} rows per step (oracle, all cores); "
              f"a full oracle dendrogram evaluates N(N-1)/2 pairs at this per-pair rate")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "d": d, "sample_rows": R},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------
# our path
# ------------------------------------------------------------------------------------

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def measure_arith_peaks():
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s, 2 flops per FMA) from the
    library's own microbenchmark kernels (libnnm_peaks.so), timed with CUDA events.
    Each kernel runs about 50-100 ms; the clocks seen meanwhile are sampled."""
    import ctypes

    from paper_1402_3789_gb300 import build
    build.build()
    lib = ctypes.CDLL(build.peaks_library_path())
    out = {}
    import torch
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    for name, fn, iters in (("fp32_tflops", lib.nnm_peak_fp32, 20000), ("fp64_tflops", lib.nnm_peak_fp64, 400)):
        fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        fn.restype = ctypes.c_int
        best = 0.0
        for _ in range(3):
            tf, ms = ctypes.c_double(), ctypes.c_double()
            if fn(8, iters, ctypes.byref(tf), ctypes.byref(ms)) != 0:
                break
            if ms.value < 40.0:   # lengthen short runs so that launch overheads vanish
                iters = int(iters * 60.0 / max(ms.value, 1e-3))
                continue
            best = max(best, tf.value)
        out[name] = best
    clocks = sampler.stop()
    out["sm_mhz"] = clocks.get("sm_mhz")
    out["method"] = ("own FMA-chain kernels (8 independent chains per thread, 8 blocks of 256 threads per SM), "
                     "CUDA events, best of 3 runs of >= 40 ms; flops = 2 per FMA")
    return out


KERNEL_SOURCES = ["paper_1402_3789_gb300/csrc/sweep_tc.cu", "paper_1402_3789_gb300/csrc/select.cuh",
                  "paper_1402_3789_gb300/csrc/nnm_internal.cuh"]


def captured_traffic(precision, N):
    """DRAM bytes per launch of the sweep from a committed ncu capture (profiles/*_dram.md)
    of this precision and N, if the kernel's sources are still the ones captured."""
    import glob
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    sha = h.hexdigest()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*_dram.md")):
        kv = {}
        with open(path) as fh:
            for ln in fh:
                ln = ln.strip()
                if ":" in ln and ln.split(":", 1)[0] in ("precision", "N", "kernel_sources_sha1", "dram_bytes_per_launch"):
                    k, v = ln.split(":", 1)
                    kv[k] = v.strip()
        if kv.get("precision") == precision and kv.get("N") == str(N) and kv.get("kernel_sources_sha1") == sha:
            return float(kv["dram_bytes_per_launch"]), os.path.basename(path)
    return None, None


def run_ours(args, world, rank, local):
    import torch

    from paper_1402_3789_gb300 import nnm
    from paper_1402_3789_gb300.inputs import WORKLOADS, make

    nnm.load_library()
    w = WORKLOADS[args.workload]
    X = make(args.workload, n=args.n)
    N, d = X.shape
    restr = dict(w.restrictions)
    Xd = torch.from_numpy(X).cuda()
    stream = torch.cuda.current_stream()

    def step(precision):
        ctx = nnm.nnm_create(Xd, precision=precision)
        try:
            res = nnm.nnm_cluster(ctx, restr)
            st = nnm.nnm_get_stats(ctx)
            st["ms_prep"] = st["ms_prep"]
            return st, res
        finally:
            nnm.nnm_destroy(ctx)

    arith = measure_arith_peaks() if not args.no_peaks else {}
    for _ in range(args.warmup):
        step(args.precision)
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    last = None
    for _ in range(args.steps):
        st, last = step(args.precision)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    elapsed_ms = max_over_ranks(e0.elapsed_time(e1), world)
    ms_per_step = elapsed_ms / args.steps
    pairs = N * (N - 1) / 2
    value = world * pairs / (ms_per_step / 1e3) / 1e9

    # roofline of the dominant kernel: the all-pairs candidate sweep
    peaks, peak_kind = load_peaks()
    sweep_ms = statistics.mean(s["sweep_ms_per_launch_full"] for s in stats)
    # the work one launch does: the pairs of the tiles it evaluated (the bounding-sphere
    # and landmark tests skip the others); the whole matrix gives the effective rate beside it
    sweep_pairs = statistics.mean(s["full_sweep_pairs_computed"] for s in stats)
    all_pairs = stats[-1]["full_sweep_pairs"]
    kpad = stats[-1]["k_pad"]
    kpad1 = 16 * ((d + 6 + 15) // 16)   # K of the one-term 16-bit form (32 at d = 25)
    if args.precision == "fp32":
        per_pair = 3 * d
        peak = arith.get("fp32_tflops") or 152 * 128 * 2 * (clocks.get("sm_mhz") or 1447.0) * 1e6 / 1e12
        roof = {"bound": "alu", "peak_source": ("measured FP32 FMA throughput (own microbenchmark, "
                                                f"{arith.get('sm_mhz')} MHz median)" if arith.get("fp32_tflops")
                                                else "152 SMs x 128 FP32 lanes x 2 x median SM clock")}
    else:
        # the method's work per pair is one K = kpad1 product (2 kpad1 MMA flops); the split
        # form issues 3x that on the tensor pipe for precision, reported as the pipe's occupancy
        per_pair = 2 * kpad1
        peak = peaks.get("bf16_tflops_sustained", 1700.0)   # same rate for fp16 operands
        roof = {"bound": "tensor", "peak_source": f"bf16_tflops_sustained ({peak_kind})"}
    flops = sweep_pairs * per_pair
    achieved = flops / (sweep_ms / 1e3) / 1e12
    traffic, traffic_src = captured_traffic(args.precision, N)
    if traffic is not None:
        roof["traffic_source"] = f"profiles/{traffic_src} (ncu, dram__bytes_read.sum + dram__bytes_write.sum)"
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                 "kernel": "k_sweep_tc" if args.precision != "fp32" else "k_sweep_fp32",
                 "algorithmic_flops_per_launch": flops, "flops_per_pair": per_pair,
                 "pairs_per_launch": sweep_pairs, "pairs_full_matrix": all_pairs,
                 "effective_tflops_full_matrix": all_pairs * per_pair / (sweep_ms / 1e3) / 1e12,
                 "launch_ms": sweep_ms})
    if args.precision != "fp32":
        pipe = sweep_pairs * 2 * kpad / (sweep_ms / 1e3) / 1e12
        roof.update({"tensor_pipe_flops_per_pair": 2 * kpad, "tensor_pipe_tflops": pipe,
                     "tensor_pipe_frac": pipe / peak})
    # the binary64 re-rank against the measured FP64 peak: 3d binary64 operations per
    # re-ranked pair (d subtractions, d products, d additions)
    rr_ms = statistics.mean(s["ms_rerank"] for s in stats)
    rr_flops = statistics.mean(s["rerank_pairs"] for s in stats) * 3 * d
    rerank_roof = {"bound": "fp64", "phase_ms": rr_ms, "fp64_flops": rr_flops,
                   "achieved_tflops": rr_flops / (rr_ms / 1e3) / 1e12 if rr_ms > 0 else None,
                   "peak_tflops": arith.get("fp64_tflops"),
                   "note": "whole re-rank phase (selections, compaction and the binary64 distances)"}
    if arith.get("fp64_tflops") and rr_ms > 0:
        rerank_roof["frac"] = rerank_roof["achieved_tflops"] / arith["fp64_tflops"]

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16": "bf16+f64", "bf16x3": "bf16x3+f64", "fp16": "f16+f64",
                      "fp32": "f32+f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "d": d, "precision": args.precision,
                       "restrictions": restr, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (X and operands > 129 MB)" if N * d * 4 > 129e6
                       else "inputs smaller than L2"},
            "time_to_dendrogram_ms": ms_per_step,
            "phases_ms": {k: statistics.mean(s[k] for s in stats) for k in
                          ("ms_prep", "ms_sweep", "ms_rerank", "ms_rounds", "ms_sort", "ms_restrict", "ms_labels")},
            "rounds": stats[-1]["rounds"], "rows_rescanned": stats[-1]["rows_rescanned"],
            "rows_overflowed": stats[-1]["rows_overflowed"], "rerank_pairs": stats[-1]["rerank_pairs"],
            "max_candidates_per_row": stats[-1]["max_candidates"],
            "tiles_skipped": stats[-1]["tiles_skipped"], "tiles_swept": stats[-1]["tiles_swept"],
            "max_abs_err_vs_fp64": max(s["max_abs_err"] for s in stats),
            "max_rel_err_vs_fp64": max(s["max_rel_err"] for s in stats),
            "n_merges": last.n_merges, "n_clusters": last.n_clusters,
            "kernel_rate_gpairs": stats[-1]["pairs_evaluated"] / 2 / (statistics.mean(s["ms_sweep"] for s in stats) / 1e3) / 1e9,
            "roofline": roof, "rerank_roofline": rerank_roof, "peaks_measured": arith, "clocks": clocks,
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats))}

    # the other precisions named by --compare, one timed step each after one untimed step
    # (the first use of a precision's kernels pays their lazy module loading)
    comp = {}
    for p in [c for c in args.compare.split(",") if c and c != args.precision]:
        step(p)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        st, _ = step(p)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        comp[p] = {"time_to_dendrogram_ms": ms, "value": pairs / (ms / 1e3) / 1e9, "sweep_ms_full": st["sweep_ms_per_launch_full"],
                   "rounds": st["rounds"], "rows_rescanned": st["rows_rescanned"],
                   "rows_overflowed": st["rows_overflowed"], "tiles_swept": st["tiles_swept"],
                   "tiles_skipped": st["tiles_skipped"], "max_rel_err_vs_fp64": st["max_rel_err"]}
    if comp:
        line["compare"] = comp

    # end to end through the C ABI from host memory (nnm_cluster_host: the library copies X
    # to the device, clusters, and copies merges and labels back); the page-locked host
    # buffers are allocated before the timed region
    if not args.no_e2e:
        Xh = torch.from_numpy(X).pin_memory()
        mh = torch.empty(max(N - 1, 1) * 32, dtype=torch.uint8).pin_memory()
        lh = torch.empty(N, dtype=torch.int32).pin_memory()
        nnm.cluster_host(Xh, restr, precision=args.precision, merges_out=mh, labels_out=lh)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        nm = 0
        for _ in range(args.steps):
            merges, labels, K = nnm.cluster_host(Xh, restr, precision=args.precision, merges_out=mh, labels_out=lh)
            nm = merges.shape[0]
        t1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(t0.elapsed_time(t1), world) / args.steps
        line["e2e"] = {"value": world * pairs / (e2e_ms / 1e3) / 1e9, "unit": UNIT,
                       "h2d_bytes_per_step": N * d * 4, "d2h_bytes_per_step": N * 4 + nm * 32, "ms_per_step": e2e_ms,
                       "api": "nnm_cluster_host (C ABI, page-locked host buffers)"}

    if rank == 0 and world == 1 and not args.no_cpu:
        rate, R, dt, cores = oracle_pair_rate(X, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"exact binary64 1-NN of {R} sampled rows against all {N} rows "
                                          f"({dt:.1f} s); a full oracle dendrogram evaluates N(N-1)/2 pairs "
                                          f"at this per-pair rate"}
    if rank == 0:
        print(json.dumps(line), flush=True)


BATCHED = "nnm_batched512"


def run_batched(args, world, rank):
    """Many independent instances of uneven N and d in one batched context (one pass of
    each kernel over all of them); the one-context-per-instance loop is timed beside it.
    Every instance is resident on the device before the timed region."""
    import torch

    from paper_1402_3789_gb300 import nnm
    from paper_1402_3789_gb300.inputs import batched_instances

    nnm.load_library()
    inst = batched_instances()
    Xs = [torch.from_numpy(x).cuda() for x in inst]
    pairs = sum(x.shape[0] * (x.shape[0] - 1) / 2 for x in inst)
    stream = torch.cuda.current_stream()

    def step_batched(precision):
        ctx = nnm.nnm_create_batched(Xs, precision=precision)
        try:
            res = nnm.nnm_cluster(ctx, {})
            st = nnm.nnm_get_stats(ctx)
            return st, res
        finally:
            nnm.nnm_destroy(ctx)

    def step_loop(precision):
        for Xd in Xs:
            ctx = nnm.nnm_create(Xd, precision=precision)
            try:
                nnm.nnm_cluster(ctx, {})
            finally:
                nnm.nnm_destroy(ctx)

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = [fn(args.precision) for _ in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, out

    for _ in range(args.warmup):
        step_batched(args.precision)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    ms, out = timed(step_batched, args.steps)
    barrier(world)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, world)
    st, res = out[-1]
    loop_ms, _ = timed(step_loop, 1)
    # the autotuned form: one batched context per (N, d) bucket with the tuned setting of
    # that bucket (paper_1402_3789_gb300/tuning/gb300_batched.json), buckets concurrently
    from paper_1402_3789_gb300 import autotune
    tuning = autotune.load_tuning()
    tuned_ms = None
    if tuning:
        autotune.run(Xs, {}, tuning)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            autotune.run(Xs, {}, tuning)
        torch.cuda.synchronize()
        tuned_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world)
    line = {"metric": "G pair-distances/s, 512 independent dendrograms in one batched context",
            "value": world * pairs / (ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16": "bf16+f64", "bf16x3": "bf16x3+f64", "fp16": "f16+f64",
                                          "fp32": "f32+f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": BATCHED, "instances": len(inst), "rows_total": sum(x.shape[0] for x in inst),
                       "pairs_total": pairs, "precision": args.precision,
                       "parallelism": "replicas" if world > 1 else "single"},
            "phases_ms": {k: st[k] for k in ("ms_prep", "ms_sweep", "ms_rerank", "ms_rounds", "ms_sort",
                                             "ms_restrict", "ms_labels")},
            "rounds": st["rounds"], "n_clusters": res.n_clusters, "tiles_swept": st["tiles_swept"],
            "tiles_skipped": st["tiles_skipped"], "gpu_launches": int(st["kernel_launches"]) * args.steps,
            "one_context_per_instance_ms": loop_ms, "clocks": clocks}
    if tuned_ms is not None:
        line["autotuned"] = {"ms_per_step": tuned_ms, "value": world * pairs / (tuned_ms / 1e3) / 1e9,
                             "unit": UNIT, "mode": tuning.get("mode"), "global": tuning.get("global"),
                             "buckets": len(tuning.get("table", {})),
                             "note": "the tuned run (paper_1402_3789_gb300/tuning/gb300_batched.json): one "
                                     "batched context with the tuned setting, or one per (N, d) bucket "
                                     "concurrently, whichever the tuning measured faster; wall-clock per "
                                     "pass, results on the device"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == BATCHED:
        run_batched(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
