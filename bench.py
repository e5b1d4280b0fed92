"""Benchmark of the LCS hot path on GB300: one step = LCS length + traceback of one long pair.

Workload: X and Y of m = n = 65536 uniform i.i.d. DNA symbols (seeded), the LCS length and the LCS string by the
paper's tie-break (UP when c[i-1,j] >= c[i,j-1]); every step runs all stages (alphabet and match masks, the table
fill writing the 1-bit direction bitmap, the parallel traceback). Metric: GCUPS = m*n / seconds / 1e9.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. `value` is timed on the device with the inputs resident in HBM (CUDA events around each step
on the launching stream; the step writes a 537 MB bitmap, more than the 129 MB L2, and an explicit L2 flush runs
between timed steps outside the events). `e2e` times the same step through the host-buffer call lcs_traceback
(host->device copy of X and Y, device->host copy of the result, inside the timed region). `--impl reference` times
the CPU oracle instead, on the host cores, on a bounded sample of the same workload (the first rows of X).
Under torchrun (N > 1) every rank runs its own replica of the step on its own GPU (the single-pair path does not
shard); value = total cells of all ranks / the slowest rank's time. Before timing, the library's autotuner picks the
fill configuration on the pair (--no-autotune keeps the default).

Other workloads (--workload): batch (10000 pairs in one persistent launch; split over ranks by pair under
torchrun), long (262144^2, length only), serve (Poisson request streams through the server), table1 (the shapes of
the paper's Table 1 against the serial and the multi-threaded CPU oracle).
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = N = 65536
SIGMA = 4
WORKLOAD = "single pair, X and Y uniform DNA (sigma=4), m=n=65536: LCS length + traceback string"
WORKLOAD_MUTATED = ("single pair, DNA (sigma=4), m=n=65536, Y = X with 10% substitutions, 2% insertions, 2% deletions: "
                    "LCS length + traceback string")


def pair_inputs(args, gen):
    """The pair workload's strings: independent uniform DNA (default) or a mutated copy (--variant mutated)."""
    if getattr(args, "variant", "uniform") == "mutated":
        x, y = gen.pair_mutated(max(args.m, args.n), SIGMA, seed=gen.BASE_SEED + 1)
        return x[: args.m], y[: args.n], WORKLOAD_MUTATED
    x, y = gen.pair_uniform(args.m, args.n, SIGMA, seed=gen.BASE_SEED + 1)
    return x, y, WORKLOAD
METRIC = "LCS GCUPS on 1 GB300 vs int-ALU roofline; serve p50/p99 latency vs per-pair"
HBM_FALLBACK_GBS = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, name in enumerate(names[1:], start=5):
                if p[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(x, y, budget_rows: int):
    """Times the oracle (LCS-length + Print-LCS) on the first budget_rows rows of X against all of Y."""
    from oracle import oracle
    oracle.build()
    xs = x[:budget_rows]
    t0 = time.perf_counter()
    s = oracle.lcs_traceback(xs, y)
    dt = time.perf_counter() - t0
    return len(xs) * len(y) / dt / 1e9, dt, len(s)


def cpu_oracle_par_sample(x, y, budget_rows: int, threads: int):
    """Times the multi-threaded oracle (column blocks over host threads) on the same sample."""
    from oracle import oracle
    oracle.build()
    xs = x[:budget_rows]
    t0 = time.perf_counter()
    oracle.lcs_traceback_par(xs, y, threads)
    dt = time.perf_counter() - t0
    return len(xs) * len(y) / dt / 1e9, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    from paper_1306_4627_gb300 import gen
    x, y, workload = pair_inputs(args, gen)
    rows = args.ref_rows
    for _ in range(args.warmup):
        cpu_oracle_sample(x, y, max(8, rows // 8))
    times = []
    for _ in range(args.steps):
        g, dt, _ = cpu_oracle_sample(x, y, rows)
        times.append(dt)
    cells = rows * N
    value = cells / float(np.mean(times)) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(times)) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload, "m": M, "n": N, "sigma": SIGMA},
        "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": 1, "kind": "oracle",
                         "sample": f"first {rows} rows of X against all {N} columns of Y per step "
                                   f"({cells:.3g} cells), LCS-length with table b + Print-LCS"},
        "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def flush_l2(buf):
    buf.add_(1)  # writes 256 MiB (> 129 MB L2)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The slowest rank's time (a barrier first, then a MAX all-reduce); the value itself on one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1306_4627_gb300 import gen, lcs

    x_np, y_np, workload = pair_inputs(args, gen)
    dev = torch.device("cuda", local)
    x = torch.from_numpy(x_np.copy()).to(dev)
    y = torch.from_numpy(y_np.copy()).to(dev)
    out = torch.empty(min(M, N), dtype=torch.uint8, device=dev)
    out_len = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    ctx = lcs.Context(local)
    stream = torch.cuda.Stream(device=dev)
    tuned = None
    if not args.no_autotune:  # the library's autotuner picks the fill configuration on this pair, before timing
        tuned = ctx.autotune_dev(x, y, traceback=True, stream=stream)
    ctx.set_profiling(True)

    def step():
        ctx.traceback_dev(x, y, out, out_len, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
            flush_l2(flush)
    torch.cuda.synchronize()
    ctx.sync()
    L = int(out_len.item())

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fill_ms, trace_ms, prep_ms = [], [], []
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
            p = ctx.last_profile()  # waits for this step's stage events
            fill_ms.append(p["fill_ms"])
            trace_ms.append(p["trace_ms"])
            prep_ms.append(p["prep_ms"])
            flush_l2(flush)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ctx.sync()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = max_over_ranks(float(np.mean(step_ms)), dist, dev)
    cells = M * N
    value = ws * cells / (t_ms * 1e-3) / 1e9

    # end to end through the host-buffer call (pinned host inputs, result copied back inside the timed region)
    xh = torch.from_numpy(x_np.copy()).pin_memory()
    yh = torch.from_numpy(y_np.copy()).pin_memory()
    ctx.set_profiling(False)
    e2e_times = []
    s_out = b""
    for k in range(0 if args.no_e2e else args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s_out = ctx.traceback(xh.numpy(), yh.numpy())
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e_times.append(dt)
    # median of the timed calls (one slow call, e.g. a host-side hiccup, moves the mean by its whole excess); the
    # mean is reported next to it
    e2e_s = max_over_ranks(float(np.median(e2e_times)) if e2e_times else float("nan"), dist, dev)
    e2e_mean_s = max_over_ranks(float(np.mean(e2e_times)) if e2e_times else float("nan"), dist, dev)
    assert args.no_e2e or len(s_out) == L

    # roofline of the dominant kernel (the fill): algorithmic bytes = the 1-bit-per-cell direction bitmap
    hbm, src = peaks()
    f_ms = float(np.mean(fill_ms))
    alg_bytes = cells / 8
    achieved = alg_bytes / (f_ms * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "fill_traffic.json")
    if os.path.exists(tfile):
        try:
            with open(tfile) as f:
                traffic = json.load(f).get("bytes_per_launch_65536")
        except Exception:
            traffic = None

    cpu = cpu_par = None
    if rank == 0 and not args.no_cpu:
        g, dt, _ = cpu_oracle_sample(x_np, y_np, args.cpu_rows)
        cpu = {"value": g, "unit": "GCUPS", "cores": 1, "kind": "oracle",
               "sample": f"first {args.cpu_rows} rows of X against all {N} columns of Y "
                         f"({args.cpu_rows * N:.3g} cells, {dt:.1f} s), LCS-length with table b + Print-LCS"}
        cores = os.cpu_count() or 1
        gp, dtp = cpu_oracle_par_sample(x_np, y_np, args.cpu_rows, cores)
        cpu_par = {"value": gp, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                   "sample": f"the same {args.cpu_rows} rows, the multi-threaded oracle (the paper's column-block "
                             f"parallel fill, {dtp:.2f} s)"}
    launches_per_step = 9  # k_alphabet, k_peq, k_xoff, k_fill, k_corr_pre, k_corr_cols, k_walk, k_chain, k_finalize
    line = {
        "metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload, "m": M, "n": N, "sigma": SIGMA, "seed": gen.BASE_SEED + 1,
                   "lcs_length": L, "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                   "l2": "explicit 256 MiB L2 flush between timed steps (outside the events); each step also "
                         "writes a 537 MB bitmap"},
        "stages_ms": {"prep": float(np.mean(prep_ms)), "fill": f_ms, "trace": float(np.mean(trace_ms))},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "kernel": "k_fill<8,true>", "peak_source": src,
                     "note": "algorithmic bytes = m*n/8 (1-bit direction bitmap) per launch"},
        "roofline_alu": alu_line(cells, 6, f_ms, clocks, "k_fill<8,true> (traceback mode)"),
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_par,
        "e2e": {"value": ws * cells / e2e_s / 1e9, "unit": "GCUPS", "stat": "median of the timed calls",
                "value_from_mean": ws * cells / e2e_mean_s / 1e9, "h2d_bytes_per_step": M + N,
                "d2h_bytes_per_step": 8 + L},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "fill_config": tuned or ctx.get_fill_config(traceback=True),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def alu_peak_tops(sm_mhz: float, sms: int = 152) -> float:
    """INT32 ALU peak from unit counts and clock: 64 INT32 lanes per SM per clock (LOP3/IADD3) x SMs x clock."""
    return sms * 64 * sm_mhz * 1e6 / 1e12


def alu_line(cells: int, ops_per_word: int, kernel_ms: float, clocks: dict, kernel: str) -> dict:
    """The fill kernel against the INT32 ALU roofline: algorithmic work = ops_per_word INT32 operations per 32 cells
    (4 for the row update, 6 with the direction bitmap), over the kernel's event-timed duration."""
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = alu_peak_tops(sm_mhz)
    achieved = cells / 32 * ops_per_word / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu (dependency chain in practice)", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak, "kernel": kernel, "ops_per_32_cells": ops_per_word,
            "note": "peak = 152 SMs x 64 INT32/clk x sampled SM clock; the single-pair fill is a wavefront whose "
                    "serial chain of steps, not the ALU, sets its time"}


def run_batch_workload(args):
    """10000 independent pairs (m, n log-uniform in [64, 4096]; alphabet 4 for half, 20 for the other half),
    lengths only, one persistent launch per step; plus the same pairs as sequential single-pair launches. Under
    torchrun the batch is split over the ranks by pair (cells balanced, no data exchanged) and value = all cells /
    the slowest rank's time."""
    import torch
    from paper_1306_4627_gb300 import gen, lcs, shard
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    all_pairs = gen.batch_pairs()
    total_cells = int(sum(len(x) * len(y) for x, y in all_pairs))
    parts = shard.partition_pairs([len(x) for x, _ in all_pairs], [len(y) for _, y in all_pairs], ws)
    pairs = [all_pairs[k] for k in parts[rank]]
    xs = np.concatenate([x for x, _ in pairs])
    ys = np.concatenate([y for _, y in pairs])
    xo = np.zeros(len(pairs) + 1, np.int64)
    yo = np.zeros(len(pairs) + 1, np.int64)
    xo[1:] = np.cumsum([len(x) for x, _ in pairs])
    yo[1:] = np.cumsum([len(y) for _, y in pairs])
    cells = int(sum(len(x) * len(y) for x, y in pairs))
    dxs, dys = torch.from_numpy(xs).to(dev), torch.from_numpy(ys).to(dev)
    dxo, dyo = torch.from_numpy(xo).to(dev), torch.from_numpy(yo).to(dev)
    out = torch.zeros(len(pairs), dtype=torch.int64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    ctx = lcs.Context(local)
    stream = torch.cuda.Stream(device=dev)
    tuned = None
    if not args.no_autotune:  # the library's batch autotuner picks words per lane, job height and blocks per SM
        tuned = ctx.autotune_batch_dev(dxs, dxo, dys, dyo, len(pairs), out, stream=stream)
    for _ in range(args.warmup):
        ctx.batch_dev(dxs, dxo, dys, dyo, len(pairs), out, stream=stream)
    ctx.sync()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    sampler.start()
    time.sleep(0.3)
    # per call (the plan is reused and the launches replay as a CUDA graph): CUDA events on the call's stream
    tot = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush_l2(flush)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.batch_dev(dxs, dxo, dys, dyo, len(pairs), out, stream=stream)
        e1.record(stream)
        e1.synchronize()
        tot.append(e0.elapsed_time(e1) * 1e-3)
    # stage split with the context's stage events (direct launches)
    ctx.set_profiling(True)
    kern, prep = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush_l2(flush)
        ctx.batch_dev(dxs, dxo, dys, dyo, len(pairs), out, stream=stream)
        p = ctx.last_profile()
        kern.append(p["fill_ms"])
        prep.append(p["prep_ms"])
    ctx.set_profiling(False)
    clocks = sampler.stop()
    ctx.sync()
    # host-buffer end to end (concatenated pinned host buffers and offsets, as a caller holds them)
    xs_h = torch.from_numpy(xs).pin_memory().numpy()
    ys_h = torch.from_numpy(ys).pin_memory().numpy()
    e2e = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ctx.batch_concat(xs_h, xo, ys_h, yo)
        if k >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    # sequential per-pair launches on a sample of the pairs (lcs_length_dev, one pair at a time)
    sample = list(range(0, len(pairs), max(1, len(pairs) // args.seq_sample)))
    dx1 = [torch.from_numpy(pairs[i][0].copy()).to(dev) for i in sample]
    dy1 = [torch.from_numpy(pairs[i][1].copy()).to(dev) for i in sample]
    o1 = torch.zeros(1, dtype=torch.int64, device=dev)
    for a, b in zip(dx1[:5], dy1[:5]):
        ctx.length_dev(a, b, o1)
    ctx.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a, b in zip(dx1, dy1):
        ctx.length_dev(a, b, o1)
    ctx.sync()
    seq_s = time.perf_counter() - t0
    seq_cells = sum(len(pairs[i][0]) * len(pairs[i][1]) for i in sample)
    t_ms = max_over_ranks(float(np.median(tot)) * 1e3, dist, dev)
    k_ms = max_over_ranks(float(np.median(kern)), dist, dev)
    e2e_s = max_over_ranks(float(np.median(e2e)), dist, dev)
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = alu_peak_tops(sm_mhz)
    achieved = total_cells / ws / 32 * 4 / (k_ms * 1e-3) / 1e12  # per GPU (the shards are cell-balanced)
    line = {
        "metric": METRIC, "value": total_cells / (t_ms * 1e-3) / 1e9, "unit": "GCUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batch: 10000 pairs, m and n log-uniform in [64, 4096], sigma 4 (half) and 20 (half), "
                               "lengths only", "cells": total_cells, "pairs": len(all_pairs),
                   "parallelism": f"pairs split over {ws} ranks, cells balanced" if ws > 1 else "1 GPU",
                   "l2": "explicit 256 MiB L2 flush before every timed call (outside the events)"},
        "batch_config": tuned or ctx.get_batch_config(),
        "stages_ms": {"prep": float(np.median(prep)), "batch_kernel": k_ms},
        "kernel_gcups": total_cells / (k_ms * 1e-3) / 1e9,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_batch_main",
                     "note": "algorithmic work = 4 INT32 ops per 32 cells; peak = 152 SMs x 64 INT32/clk x sampled "
                             "SM clock"},
        "sequential_per_pair": {"gcups": seq_cells / seq_s / 1e9, "pairs_timed": len(sample),
                                "speedup_of_batch": (total_cells / ws / (t_ms * 1e-3)) / (seq_cells / seq_s),
                                "note": "lcs_length_dev per pair, back to back, same GPU"},
        "e2e": {"value": total_cells / e2e_s / 1e9, "unit": "GCUPS", "stat": "median of the timed calls",
                "h2d_bytes_per_step": int(xs.nbytes + ys.nbytes), "d2h_bytes_per_step": 8 * len(pairs)},
        "gpu_launches": 3 * args.steps, "clocks": clocks,  # k_batch_prep, k_batch_main, k_batch_combine per call
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def run_long_workload(args):
    """One length-only pair of m = n = 262144 (alphabet 4 and 20)."""
    import torch
    from paper_1306_4627_gb300 import gen, lcs
    dev = torch.device("cuda", 0)
    res = {}
    ctx = lcs.Context(0)
    ctx.set_profiling(True)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    for sigma in (4, 20):
        x, y = gen.pair_uniform(262144, 262144, sigma, seed=gen.BASE_SEED + 2)
        dx, dy = torch.from_numpy(x.copy()).to(dev), torch.from_numpy(y.copy()).to(dev)
        out = torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(args.warmup):
            ctx.length_dev(dx, dy, out, stream=stream)
        ctx.sync()
        ts, fs = [], []
        for _ in range(args.steps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush_l2(flush)
            ev0.record(stream)
            ctx.length_dev(dx, dy, out, stream=stream)
            ev1.record(stream)
            p = ctx.last_profile()
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1))
            fs.append(p["fill_ms"])
        res[sigma] = (float(np.median(ts)), float(np.median(fs)), int(out.item()))
    clocks = sampler.stop()
    cells = 262144 ** 2
    t4 = res[4][0]
    line = {
        "metric": METRIC, "value": cells / (t4 * 1e-3) / 1e9, "unit": "GCUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t4, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": "single pair, length only, m=n=262144, sigma 4 (value) and 20",
                   "sigma20_gcups": cells / (res[20][0] * 1e-3) / 1e9, "lcs_length": {4: res[4][2], 20: res[20][2]},
                   "l2": "explicit 256 MiB L2 flush before every timed call (outside the events)"},
        "stages_ms": {"fill_sigma4": res[4][1], "fill_sigma20": res[20][1]},
        "roofline": alu_line(cells, 4, res[4][1], clocks, "k_fill<8,false> (length only, meet in the middle)"),
        # per call: k_alphabet, k_peq, k_xoff, k_fill, k_combine_pre, k_combine_min, k_combine_fin; both alphabets
        "gpu_launches": 2 * 7 * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_serve_workload(args):
    """Poisson request streams at swept rates: m and n log-uniform in [32, 65536], alphabet 4, 20 or 256, 20%
    traceback. Latency (submit to result) is measured by the server; each rate also records the service time of
    the same requests run one by one through the single-pair calls (the per-pair baseline)."""
    from paper_1306_4627_gb300 import gen, lcs
    ctx = lcs.Context(0)
    rates = [float(r) for r in args.rates.split(",")]
    out_rates = []
    for rate in rates:
        reqs = gen.serve_requests(rate=rate, count=args.serve_count, seed=gen.BASE_SEED + 4)
        cells = sum(len(r["x"]) * len(r["y"]) for r in reqs)
        srv = lcs.Server(ctx, pair_workers=args.pair_workers)
        # warm the workers' buffers with a few requests
        for r in reqs[:8]:
            srv.wait(srv.submit(r["x"], r["y"], traceback=r["traceback"]), timeout_s=60.0)
        tickets = []
        t0 = time.perf_counter()
        for r in reqs:
            due = t0 + r["t"] - reqs[0]["t"]
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                if due - now > 2e-4:
                    time.sleep((due - now) * 0.5)
            while True:
                rc, t = srv.try_submit(r["x"], r["y"], traceback=r["traceback"])
                if rc == lcs.OK:
                    break
                time.sleep(1e-4)  # back-pressure: retry
            tickets.append(t)
        lat = []
        for t in tickets:
            res = srv.wait(t, timeout_s=600.0)
            lat.append(res["latency_s"])
        wall = time.perf_counter() - t0
        srv.close()
        lat = np.array(lat)
        out_rates.append({"rate_per_s": rate, "requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                          "p99_ms": float(np.percentile(lat, 99) * 1e3), "gcups": cells / wall / 1e9,
                          "offered_gcups": cells / (reqs[-1]["t"] - reqs[0]["t"]) / 1e9, "wall_s": wall})
        print(json.dumps({"serve_rate": out_rates[-1]}), file=sys.stderr, flush=True)
    # per-pair baseline: the same request mix, one call at a time (service time of each)
    reqs = gen.serve_requests(rate=1000.0, count=min(args.serve_count, 1000), seed=gen.BASE_SEED + 4)
    svc = []
    for r in reqs:
        t1 = time.perf_counter()
        (ctx.traceback if r["traceback"] else ctx.length)(r["x"], r["y"])
        svc.append(time.perf_counter() - t1)
    svc = np.array(svc)
    best = max(out_rates, key=lambda d: d["gcups"])
    line = {
        "metric": METRIC, "value": best["gcups"], "unit": "GCUPS", "n_gpus": 1, "steps": len(rates),
        "warmup": 1, "ms_per_step": best["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals, m,n log-uniform [32, 65536], sigma 4/20/256, 20% traceback",
                   "requests_per_rate": args.serve_count, "pair_workers": args.pair_workers or 8},
        "rates": out_rates,
        "per_pair_baseline": {"p50_ms": float(np.percentile(svc, 50) * 1e3), "p99_ms": float(np.percentile(svc, 99) * 1e3),
                              "gcups": sum(len(r["x"]) * len(r["y"]) for r in reqs) / svc.sum() / 1e9,
                              "note": "each request alone through lcs_length / lcs_traceback, one at a time"},
    }
    print(json.dumps(line), flush=True)
    ctx.close()


# The paper's experiment (Table 1): parent length M (rows, X) x child length N (columns, Y), DNA strings.
TABLE1_SHAPES = [(10, 5), (100, 10), (200, 30), (500, 80), (800, 100), (1000, 150), (2000, 200), (5000, 200),
                 (5000, 400), (5000, 800), (5000, 1000), (10000, 1000), (10000, 1500)]


def _time_reps(fn, min_s: float = 0.05, max_reps: int = 200) -> float:
    """Median seconds of fn() over repetitions that add up to at least min_s (one warm call first)."""
    fn()
    ts = []
    while len(ts) < max_reps and (sum(ts) < min_s or len(ts) < 3):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def run_table1_workload(args):
    """The shapes of the paper's Table 1 with uniform DNA strings: per shape the traceback through the host-buffer
    call (length and LCS string, copies included), its device time, the serial oracle on one core and the
    multi-threaded oracle (the paper's column-block parallel fill) on all host cores. The paper's speedup column
    is parallel CPU time against serial CPU time; the GPU columns are this library."""
    from oracle import oracle
    from paper_1306_4627_gb300 import gen, lcs
    oracle.build()
    cores = os.cpu_count() or 1
    ctx = lcs.Context(0)
    rows, tot_cells, tot_gpu, tot_par = [], 0, 0.0, 0.0
    for k, (m, n) in enumerate(TABLE1_SHAPES):
        x, y = gen.pair_uniform(m, n, 4, seed=gen.BASE_SEED + 100 + k)
        s_gpu = ctx.traceback(x, y)
        parity = s_gpu == oracle.lcs_traceback(x, y) == oracle.lcs_traceback_par(x, y, cores)
        t_gpu = _time_reps(lambda: ctx.traceback(x, y))
        ctx.set_profiling(True)
        dev, stages = [], []
        for _ in range(max(3, args.steps)):
            ctx.traceback(x, y)
            p = ctx.last_profile()
            dev.append(p["total_ms"])
            stages.append((p["prep_ms"], p["fill_ms"], p["trace_ms"]))
        ctx.set_profiling(False)
        st = np.median(np.array(stages), axis=0)
        t_cpu1 = _time_reps(lambda: oracle.lcs_traceback(x, y), min_s=0.02)
        t_cpun = _time_reps(lambda: oracle.lcs_traceback_par(x, y, cores), min_s=0.02)
        rows.append({"M": m, "N": n, "lcs_length": len(s_gpu), "parity_with_oracle": bool(parity),
                     "gpu_e2e_ms": t_gpu * 1e3, "gpu_device_ms": float(np.median(dev)),
                     "gpu_stages_ms": {"prep": float(st[0]), "fill": float(st[1]), "trace": float(st[2])},
                     "cpu_1core_ms": t_cpu1 * 1e3, f"cpu_{cores}core_ms": t_cpun * 1e3,
                     "cpu_parallel_speedup": t_cpu1 / t_cpun, "gpu_e2e_vs_cpu_1core": t_cpu1 / t_gpu})
        tot_cells += m * n
        tot_gpu += t_gpu
        tot_par += t_cpun
        print(json.dumps({"table1_shape": rows[-1]}), file=sys.stderr, flush=True)
    line = {
        "metric": METRIC, "value": tot_cells / tot_gpu / 1e9, "unit": "GCUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": 1, "ms_per_step": tot_gpu * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "the 13 shapes of the paper's Table 1 (M x N from 10x5 to 10000x1500), uniform DNA, "
                               "traceback through the host-buffer call; value = all cells / summed per-call time"},
        "sweep": rows,
        "cpu_baseline": {"value": tot_cells / tot_par / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                         "sample": "all 13 shapes, multi-threaded oracle (column blocks over host threads)"},
        "all_parity": all(r["parity_with_oracle"] for r in rows),
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    global M, N
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=16384)
    ap.add_argument("--ref-rows", type=int, default=2048)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--m", type=int, default=M, help="rows (profiling of smaller cases only)")
    ap.add_argument("--n", type=int, default=N, help="columns (profiling of smaller cases only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default fill configuration")
    ap.add_argument("--workload", default="pair", choices=["pair", "batch", "long", "serve", "table1"],
                    help="pair: the 65536^2 traceback step (default); batch: 10000 pairs; long: 262144^2 length; "
                         "serve: Poisson request streams; table1: the shapes of the paper's Table 1")
    ap.add_argument("--seq-sample", type=int, default=400, help="pairs timed as sequential single-pair launches")
    ap.add_argument("--rates", default="1000,3000,10000,30000,100000", help="serving: request rates per second")
    ap.add_argument("--serve-count", type=int, default=3000, help="serving: requests per rate")
    ap.add_argument("--pair-workers", type=int, default=0, help="serving: single-pair workers (0 = the default)")
    ap.add_argument("--variant", default="uniform", choices=["uniform", "mutated"],
                    help="pair workload: independent uniform DNA (default) or Y a mutated copy of X")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    M, N = args.m, args.n
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_workload(args)
    elif args.workload == "long":
        run_long_workload(args)
    elif args.workload == "serve":
        run_serve_workload(args)
    elif args.workload == "table1":
        run_table1_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
