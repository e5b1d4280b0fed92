"""Benchmark of the LCS hot path on GB300. The headline step = LCS length + traceback of one 65536^2 pair.

Headline workload: X and Y of m = n = 65536 uniform i.i.d. DNA symbols (seeded), the LCS length and the LCS string
by the paper's tie-break (UP when c[i-1,j] >= c[i,j-1]); every step runs all stages (alphabet and match masks, the
table fill writing the 1-bit direction bitmap, the parallel traceback). Metric: GCUPS = m*n / seconds / 1e9.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload all|pair|batch|long|serve|table1]

Prints one JSON line. `value` is timed on the device with the inputs resident in HBM (CUDA events around each of
the K steps on the launching stream; the step writes a 537 MB bitmap, more than the 129 MB L2, and an explicit L2
flush runs between timed steps outside the events). `e2e` times the same step through the host-buffer call
lcs_traceback (host->device copy of X and Y, device->host copy of the result, inside the timed region).

With the default --workload all (one GPU) the line also carries, under "workloads", every other configuration of
the benchmark suite, each with a timed region of at least one second, its own clock samples, a roofline against a
ceiling measured in the same run, and a CPU-oracle baseline:
  probes              the device's INT32 rate for the fill's instruction mix and the fill step's dependency floor
  pair_2048           a 2048^2 DNA pair, length + traceback
  pair_65536_mutated  65536^2, Y = X with 10% substitutions, 2% insertions, 2% deletions, length + traceback
  long_262144         262144^2 length only, alphabets 4 and 20
  batch_10000         10000 pairs (m, n log-uniform in [64, 4096], alphabets 4 and 20) in one persistent launch
  serve               Poisson request streams at 1k-100k requests/s through the continuous-batching server
`--impl reference` times the CPU oracle instead, on the host cores, on a bounded sample of the headline workload.
Under torchrun (N > 1) every rank runs its own replica of the headline step on its own GPU (the single-pair path
does not shard); value = total cells of all ranks / the slowest rank's time; `--workload batch` splits the batch
over the ranks by pair instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The serving workload runs 18 worker streams at once (16 single-pair and 2 batch workers). With the CUDA runtime's
# default of 8 hardware work queues per process, streams share queues and the kernels of different workers wait on
# each other (measured: 3.2k against 5.5k GCUPS at saturation). 32 queues give each worker its own. This is read
# when the process first initialises CUDA, which happens later (torch is imported inside the workloads); a value
# the caller set explicitly is kept.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

M = N = 65536
SIGMA = 4
WORKLOAD = "single pair, X and Y uniform DNA (sigma=4), m=n=65536: LCS length + traceback string"
WORKLOAD_MUTATED = ("single pair, DNA (sigma=4), m=n=65536, Y = X with 10% substitutions, 2% insertions, 2% deletions: "
                    "LCS length + traceback string")
METRIC = "LCS GCUPS on 1 GB300 vs int-ALU roofline; serve p50/p99 latency vs per-pair"
HBM_FALLBACK_GBS = 6800.0
# library kernel launches per call: k_alphabet, k_xoff (masks and row offsets), k_fill, k_corr_pre, k_corr_cols,
# k_walk, k_chain, k_finalize (traceback); k_alphabet, k_xoff, k_fill and the combine (length, meet in the middle)
LAUNCHES_TRACEBACK = 8
LAUNCHES_LENGTH_SPLIT_WIDE = 6  # beyond 2048 words the combine takes three launches
LAUNCHES_LENGTH_SPLIT = 4


def pair_inputs(args, gen):
    """The pair workload's strings: independent uniform DNA (default) or a mutated copy (--variant mutated)."""
    if getattr(args, "variant", "uniform") == "mutated":
        x, y = gen.pair_mutated(max(args.m, args.n), SIGMA, seed=gen.BASE_SEED + 1)
        return x[: args.m], y[: args.n], WORKLOAD_MUTATED
    x, y = gen.pair_uniform(args.m, args.n, SIGMA, seed=gen.BASE_SEED + 1)
    return x, y, WORKLOAD


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
         "clocks_event_reasons.sw_power_cap,utilization.gpu")

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
        return self

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
        sm, mx, pw, util, reasons = [], [], [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
                pw.append(float(p[3]))
                util.append(float(p[9]) if len(p) > 9 else float("nan"))
            except ValueError:
                continue
            for k, name in enumerate(names[1:], start=5):
                if p[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(pw) if pw else None,
                "gpu_util_pct_median": float(np.nanmedian(util)) if util and not np.all(np.isnan(util)) else None}


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


def cpu_baselines_traceback(x, y, rows: int) -> tuple[dict, dict]:
    """The serial oracle on one core and the multi-threaded oracle on all host cores, on the first `rows` rows."""
    rows = min(rows, len(x))
    g, dt, _ = cpu_oracle_sample(x, y, rows)
    one = {"value": g, "unit": "GCUPS", "cores": 1, "kind": "oracle",
           "sample": f"first {rows} rows of X against all {len(y)} columns of Y ({rows * len(y):.3g} cells, "
                     f"{dt:.2f} s), LCS-length with table b + Print-LCS"}
    cores = os.cpu_count() or 1
    gp, dtp = cpu_oracle_par_sample(x, y, rows, cores)
    allc = {"value": gp, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": f"the same {rows} rows, the multi-threaded oracle (the paper's column-block parallel fill, "
                      f"{dtp:.2f} s)"}
    return one, allc


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


def timed_calls(call, stream, min_s: float = 1.0, flush=None, max_calls: int = 100000) -> list[float]:
    """Device time (ms) of each of as many back-to-back calls of `call` on `stream` as fill at least min_s seconds:
    every call bracketed by its own CUDA events on the stream, `flush` (an L2 flush) between calls outside the
    events. The count comes from three untimed calls."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        call()
        e0.record(stream)
        for _ in range(3):
            call()
        e1.record(stream)
    e1.synchronize()
    est_ms = max(e0.elapsed_time(e1) / 3.0, 1e-3)
    count = int(min(max_calls, max(3, math.ceil(min_s * 1e3 / est_ms))))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(count)]
    with torch.cuda.stream(stream):
        for a, b in evs:
            if flush is not None:
                flush()
            a.record(stream)
            call()
            b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def host_calls(call, min_s: float = 1.0, warm: int = 3, max_calls: int = 100000) -> list[float]:
    """Wall-clock seconds of each of as many back-to-back host calls as fill at least min_s seconds (after `warm`
    untimed ones)."""
    for _ in range(warm):
        call()
    ts = []
    t_end = time.perf_counter() + min_s
    while (time.perf_counter() < t_end or len(ts) < 3) and len(ts) < max_calls:
        t0 = time.perf_counter()
        call()
        ts.append(time.perf_counter() - t0)
    return ts


# ---- ceilings: measured INT32 rate and the fill's dependency floor ----------------------------------------------

def measure_probes(device: int) -> dict:
    """INT32 throughput for the fill's instruction mixes (row update: 5 instructions per word and row; with the
    traceback word: 6; plain three-input logic) and the clock cycles of one 8-row fill step's row arithmetic and carry
    shuffles alone (length and traceback mode), all on this GPU in this run."""
    from paper_1306_4627_gb300 import lcs
    sampler = ClockSampler(device).start()
    rates = {name: lcs.probe_int_rate(device, mix, 200000) for name, mix in
             (("row_update", 0), ("row_update_traceback", 1), ("lop3", 2))}
    floors = {f"rows{b}_{'traceback' if tb else 'length'}": lcs.probe_step_floor(device, b, tb, 8192)
              for b in (8, 16) for tb in (False, True)}
    mask_src = {name: lcs.probe_step_masks(device, k, 8192) for k, name in enumerate(lcs.MASK_SOURCES)}
    clocks = sampler.stop()
    return {"int_rate": rates, "step_floor_cycles": floors, "step_mask_source_cycles": mask_src, "clocks": clocks,
            "note": "int_rate: every SM full of independent chains of the mix (ops = instructions of the mix); "
                    "step_floor_cycles: one warp per SM sub-partition running only the fill's row arithmetic and "
                    "carry shuffles (plus its two bitmap stores per step in traceback mode), masks in registers; "
                    "step_mask_source_cycles: the 8-row traceback step with its masks from registers, from the "
                    "fill's shared table, or formed from two bit planes of Y's codes (byte-permuted or expanded "
                    "row codes)"}


def alu_line(cells: int, ops_per_word: int, kernel_ms: float, clocks: dict, kernel: str, probes: dict | None,
             mix: str) -> dict:
    """The fill against the INT32 ALU roofline. Work = ops_per_word instructions per 32 cells (the row update's
    5, 6 with the traceback word); peak = the measured rate of the same instruction mix on this GPU (probe), at the
    clock sampled during this workload; also the fraction of the nominal 64 INT32 lanes per SM per clock."""
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    achieved = cells / 32 * ops_per_word / (kernel_ms * 1e-3) / 1e12
    r = (probes or {}).get("int_rate", {}).get(mix)
    sms = int(r["sms"]) if r else 152
    nominal = sms * 64 * sm_mhz * 1e6 / 1e12
    if r:
        peak = r["ops_per_clk_sm"] * sms * sm_mhz * 1e6 / 1e12
        src = (f"measured: {r['ops_per_clk_sm']:.1f} instructions of the mix per SM per clock (probe, "
               f"{r['sm_clock_mhz']:.0f} MHz) x {sms} SMs x the sampled {sm_mhz:.0f} MHz")
    else:
        peak, src = nominal, "derived: 64 INT32 lanes per SM per clock (no probe)"
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "kernel": kernel, "ops_per_32_cells": ops_per_word, "peak_source": src,
            "frac_of_nominal_64_per_clk": achieved / nominal, "cells_per_s_at_peak": peak * 1e12 / ops_per_word * 32}


def dependency_line(rows: int, B: int, words: int, floor_cycles: float | None, clocks: dict, kernel_ms: float,
                    note: str) -> dict | None:
    """The chain bound of one pair's fill: (row-blocks + one step per 32-column word after the first) steps, each at
    least the measured step floor, at the sampled clock; frac = bound / measured fill time."""
    if not floor_cycles:
        return None
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    steps = math.ceil(rows / B) + (words - 1)
    bound_ms = steps * floor_cycles / (sm_mhz * 1e6) * 1e3
    return {"bound_ms": bound_ms, "measured_ms": kernel_ms, "frac": bound_ms / kernel_ms, "steps": steps,
            "floor_cycles_per_step": floor_cycles, "sm_mhz": sm_mhz, "note": note}


# ---- the headline pair and the other single-pair configurations ---------------------------------------------------

def measure_pair(dev, x_np, y_np, args, probes=None, min_s=1.0, cpu_rows=16384, label="") -> dict:
    """Length + traceback of one pair through lcs_traceback_dev: per-call device time over >= min_s seconds (L2
    flushed between calls), stage split, e2e through the host-buffer call, rooflines and the oracle baselines."""
    import torch
    from paper_1306_4627_gb300 import lcs
    m, n = len(x_np), len(y_np)
    x = torch.from_numpy(x_np.copy()).to(dev)
    y = torch.from_numpy(y_np.copy()).to(dev)
    out = torch.empty(max(1, min(m, n)), dtype=torch.uint8, device=dev)
    out_len = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    ctx = lcs.Context(dev.index)
    stream = torch.cuda.Stream(device=dev)
    tuned = ctx.autotune_dev(x, y, traceback=True, stream=stream) if not args.no_autotune else None

    def step():
        ctx.traceback_dev(x, y, out, out_len, stream=stream)

    sampler = ClockSampler(dev.index).start()
    time.sleep(0.3)
    ms = timed_calls(step, stream, min_s, flush=lambda: flush_l2(flush))
    clocks = sampler.stop()
    ctx.sync()
    L = int(out_len.item())
    ctx.set_profiling(True)
    prof = []
    for _ in range(5):
        with torch.cuda.stream(stream):
            flush_l2(flush)
        step()
        prof.append(ctx.last_profile())
    ctx.set_profiling(False)
    fill_ms = float(np.median([p["fill_ms"] for p in prof]))
    xh = torch.from_numpy(x_np.copy()).pin_memory()
    yh = torch.from_numpy(y_np.copy()).pin_memory()
    e2e = host_calls(lambda: ctx.traceback(xh.numpy(), yh.numpy()), min_s=min(min_s, 0.5))
    assert len(ctx.traceback(xh.numpy(), yh.numpy())) == L
    ctx.close()
    cells = m * n
    t = float(np.median(ms))
    hbm, src = peaks()
    bitmap_gbs = cells / 8 / (fill_ms * 1e-3) / 1e9
    one, allc = cpu_baselines_traceback(x_np, y_np, cpu_rows) if not args.no_cpu else (None, None)
    floor = ((probes or {}).get("step_floor_cycles") or {}).get("rows8_traceback")
    return {
        "workload": label, "m": m, "n": n, "lcs_length": L, "value": cells / (t * 1e-3) / 1e9, "unit": "GCUPS",
        "ms_per_call": t, "calls_timed": len(ms), "timed_s": float(np.sum(ms)) * 1e-3,
        "l2": "explicit 256 MiB L2 flush between timed calls (outside the events)",
        "stages_ms": {"prep": float(np.median([p["prep_ms"] for p in prof])), "fill": fill_ms,
                      "trace": float(np.median([p["trace_ms"] for p in prof]))},
        "roofline": {"bound": "hbm", "achieved": bitmap_gbs, "peak": hbm, "unit": "GB/s", "frac": bitmap_gbs / hbm,
                     "kernel": "k_fill (traceback)", "peak_source": src,
                     "note": "algorithmic bytes = m*n/8 (1-bit direction bitmap) per launch"},
        "roofline_alu": alu_line(cells, 6, fill_ms, clocks, "k_fill (traceback mode)", probes, "row_update_traceback"),
        "dependency_bound": dependency_line(m, 8, n // 32 + 1, floor, clocks, fill_ms,
                                            "forward fill of all m rows (the traceback needs every row's bitmap)"),
        "e2e": {"value": cells / float(np.median(e2e)) / 1e9, "unit": "GCUPS", "stat": "median of the timed calls",
                "calls": len(e2e), "h2d_bytes_per_step": m + n, "d2h_bytes_per_step": 8 + L},
        "cpu_baseline": one, "cpu_baseline_all_cores": allc,
        "gpu_launches": (LAUNCHES_TRACEBACK if m > 1024 or n > 992 else 1) * len(ms),
        "clocks": clocks, "fill_config": tuned,
    }


def run_gpu(args):
    """The headline line: K timed steps of the 65536^2 traceback (the contract's value), then at least one second
    more of the same step (clocks sampled over both), e2e, rooflines and the oracle baselines; with --workload all
    on one GPU, every other configuration under "workloads"."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1306_4627_gb300 import gen, lcs

    dev = torch.device("cuda", local)
    probes = measure_probes(local) if (ws == 1 and args.workload == "all") else None
    x_np, y_np, workload = pair_inputs(args, gen)
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
    step_ms = [a.elapsed_time(b) for a, b in evs]
    # the same step for at least one more second (clocks keep being sampled): a timed region long enough to trust
    ctx.set_profiling(False)
    sustained = timed_calls(step, stream, args.sustain_s, flush=lambda: flush_l2(flush)) if args.sustain_s > 0 else []
    clocks = sampler.stop()
    ctx.sync()
    t_ms = max_over_ranks(float(np.mean(step_ms)), dist, dev)
    cells = M * N
    value = ws * cells / (t_ms * 1e-3) / 1e9

    # end to end through the host-buffer call (pinned host inputs, result copied back inside the timed region)
    xh = torch.from_numpy(x_np.copy()).pin_memory()
    yh = torch.from_numpy(y_np.copy()).pin_memory()
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
    fill_config = tuned or ctx.get_fill_config(traceback=True)
    ctx.close()
    del x, y, out, flush
    torch.cuda.empty_cache()

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
        cpu, cpu_par = cpu_baselines_traceback(x_np, y_np, args.cpu_rows)
    floor = ((probes or {}).get("step_floor_cycles") or {}).get("rows8_traceback")
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
        "roofline_alu": alu_line(cells, 6, f_ms, clocks, "k_fill<8,true> (traceback mode)", probes,
                                 "row_update_traceback"),
        "dependency_bound": dependency_line(M, 8, N // 32 + 1, floor, clocks, f_ms,
                                            "forward fill of all m rows (the traceback needs every row's bitmap)"),
        "sustained": {"calls": len(sustained), "timed_s": float(np.sum(sustained)) * 1e-3,
                      "ms_per_step": float(np.median(sustained)) if sustained else None,
                      "value": cells / (float(np.median(sustained)) * 1e-3) / 1e9 if sustained else None,
                      "note": "the same step repeated right after the K timed steps (L2 flushed between calls, "
                              "outside the events), median per call; clocks cover both"},
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_par,
        "e2e": {"value": ws * cells / e2e_s / 1e9, "unit": "GCUPS", "stat": "median of the timed calls",
                "value_from_mean": ws * cells / e2e_mean_s / 1e9, "h2d_bytes_per_step": M + N,
                "d2h_bytes_per_step": 8 + L},
        "gpu_launches": LAUNCHES_TRACEBACK * args.steps,
        "clocks": clocks,
        "fill_config": fill_config,
    }
    if ws == 1 and args.workload == "all":
        line["workloads"] = run_all_workloads(args, dev, probes)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_all_workloads(args, dev, probes) -> dict:
    """Every other configuration of the suite on this GPU, one after the other (each frees its device memory)."""
    import torch
    from paper_1306_4627_gb300 import gen
    res = {"probes": probes}
    x, y = gen.pair_uniform(2048, 2048, 4, seed=gen.BASE_SEED + 0)
    res["pair_2048"] = measure_pair(dev, x, y, args, probes, min_s=1.0, cpu_rows=2048,
                                    label="single pair, X and Y uniform DNA (sigma=4), m=n=2048: length + traceback")
    torch.cuda.empty_cache()
    x, y = gen.pair_mutated(65536, SIGMA, seed=gen.BASE_SEED + 1)
    res["pair_65536_mutated"] = measure_pair(dev, x, y, args, probes, min_s=1.0, cpu_rows=8192, label=WORKLOAD_MUTATED)
    torch.cuda.empty_cache()
    res["long_262144"] = measure_long(args, dev, probes)
    torch.cuda.empty_cache()
    res["batch_10000"] = measure_batch(args, dev, probes)
    torch.cuda.empty_cache()
    res["serve"] = measure_serve(args, dev)
    return res


# ---- 262144^2 length only -------------------------------------------------------------------------------------------

def measure_long(args, dev, probes=None, min_s=1.0) -> dict:
    """One length-only pair of m = n = 262144 for alphabets 4 and 20 (meet in the middle: two fills of 131072 rows
    at once), each timed per call for >= min_s seconds; INT32 roofline and dependency bound of the fill; e2e through
    the host-buffer call; the oracle on a row sample (1 core) and the full-width multi-threaded oracle on more
    rows."""
    import torch
    from oracle import oracle
    from paper_1306_4627_gb300 import gen, lcs
    oracle.build()
    ctx = lcs.Context(dev.index)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    m = n = 262144
    cells = m * n
    out = {}
    for sigma in (4, 20):
        x, y = gen.pair_uniform(m, n, sigma, seed=gen.BASE_SEED + 2)
        dx, dy = torch.from_numpy(x.copy()).to(dev), torch.from_numpy(y.copy()).to(dev)
        o = torch.zeros(1, dtype=torch.int64, device=dev)
        # the library's autotuner picks the length-only fill configuration on this pair, before timing
        tuned = ctx.autotune_dev(dx, dy, traceback=False, stream=stream) if not args.no_autotune else None
        sampler = ClockSampler(dev.index).start()
        time.sleep(0.3)
        ms = timed_calls(lambda: ctx.length_dev(dx, dy, o, stream=stream), stream, min_s, flush=lambda: flush_l2(flush))
        clocks = sampler.stop()
        ctx.sync()
        L = int(o.item())
        ctx.set_profiling(True)
        fills = []
        for _ in range(5):
            ctx.length_dev(dx, dy, o, stream=stream)
            fills.append(ctx.last_profile()["fill_ms"])
        ctx.set_profiling(False)
        f_ms = float(np.median(fills))
        e2e = host_calls(lambda: ctx.length(x, y), min_s=0.3)
        t = float(np.median(ms))
        floor = ((probes or {}).get("step_floor_cycles") or {}).get("rows8_length")
        rows1, rowsn = 1024, 8192
        t0 = time.perf_counter()
        oracle.lcs_length(x[:rows1], y)
        dt1 = time.perf_counter() - t0
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        oracle.lcs_length_par(x[:rowsn], y, cores)
        dtn = time.perf_counter() - t0
        out[f"sigma{sigma}"] = {
            "value": cells / (t * 1e-3) / 1e9, "unit": "GCUPS", "lcs_length": L, "ms_per_call": t,
            "calls_timed": len(ms), "timed_s": float(np.sum(ms)) * 1e-3, "fill_ms": f_ms,
            "roofline": alu_line(cells, 5, f_ms, clocks, "k_fill<8,false> (length only, meet in the middle)", probes,
                                 "row_update"),
            "dependency_bound": dependency_line(m // 2, 8, n // 32 + 1, floor, clocks, f_ms,
                                                "meet in the middle: two chains of m/2 rows run at once"),
            "e2e": {"value": cells / float(np.median(e2e)) / 1e9, "unit": "GCUPS", "calls": len(e2e),
                    "stat": "median of the timed calls", "h2d_bytes_per_step": m + n, "d2h_bytes_per_step": 8},
            "cpu_baseline": {"value": rows1 * n / dt1 / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
                             "sample": f"LCS-length of the first {rows1} rows of X against all of Y ({dt1:.2f} s)"},
            "cpu_baseline_all_cores": {"value": rowsn * n / dtn / 1e9, "unit": "GCUPS", "cores": cores,
                                       "kind": "oracle",
                                       "sample": f"the column-block length oracle on the first {rowsn} rows "
                                                 f"({dtn:.2f} s)"},
            "gpu_launches": LAUNCHES_LENGTH_SPLIT_WIDE * len(ms),
            "clocks": clocks, "fill_config": tuned or ctx.get_fill_config(traceback=False),
        }
        del dx, dy
    ctx.close()
    return {"workload": "single pair, length only, m=n=262144, uniform over 4 and over 20 symbols",
            "l2": "explicit 256 MiB L2 flush between timed calls (outside the events)", **out}


def run_long_workload(args):
    import torch
    dev = torch.device("cuda", 0)
    probes = measure_probes(0)
    r = measure_long(args, dev, probes)
    s4 = r["sigma4"]
    line = {
        "metric": METRIC, "value": s4["value"], "unit": "GCUPS", "n_gpus": 1, "steps": s4["calls_timed"],
        "warmup": args.warmup, "ms_per_step": s4["ms_per_call"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": r["workload"], "l2": r["l2"]},
        "roofline": s4["roofline"], "e2e": s4["e2e"], "cpu_baseline": s4["cpu_baseline"],
        "gpu_launches": s4["gpu_launches"], "clocks": s4["clocks"], "detail": r, "probes": probes,
    }
    print(json.dumps(line), flush=True)


# ---- batch ----------------------------------------------------------------------------------------------------------

def measure_batch(args, dev, probes=None, min_s=1.0, ws=1, rank=0, dist=None) -> dict:
    """10000 independent pairs (m, n log-uniform in [64, 4096]; alphabet 4 for half, 20 for the other half),
    lengths only, one persistent launch per call (replayed as a CUDA graph), timed per call for >= min_s seconds with
    the L2 flushed between calls; the same pairs as sequential single-pair launches; e2e through the host call;
    the oracle on a sample of the pairs. Under torchrun each rank takes its shard (cells balanced, no exchange)."""
    import torch
    from oracle import oracle
    from paper_1306_4627_gb300 import gen, lcs, shard
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
    dxs, dys = torch.from_numpy(xs).to(dev), torch.from_numpy(ys).to(dev)
    dxo, dyo = torch.from_numpy(xo).to(dev), torch.from_numpy(yo).to(dev)
    outd = torch.zeros(len(pairs), dtype=torch.int64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)
    ctx = lcs.Context(dev.index)
    stream = torch.cuda.Stream(device=dev)
    tuned = None
    if not args.no_autotune:  # the library's batch autotuner picks words per lane, job height and blocks per SM
        tuned = ctx.autotune_batch_dev(dxs, dxo, dys, dyo, len(pairs), outd, stream=stream)
    # the timed call takes the offsets from host memory, where the caller built them (lcs_batch_dev_hoff); the
    # variant with device offsets (lcs_batch_dev) copies them back and waits before planning, timed beside it
    xo_h, yo_h = xo.astype(np.uint64), yo.astype(np.uint64)
    for _ in range(args.warmup):
        ctx.batch_dev_hoff(dxs, xo_h, dys, yo_h, len(pairs), outd, stream=stream)
    ctx.sync()
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(dev.index).start()
    time.sleep(0.3)
    tot = timed_calls(lambda: ctx.batch_dev_hoff(dxs, xo_h, dys, yo_h, len(pairs), outd, stream=stream), stream,
                      min_s, flush=lambda: flush_l2(flush))
    clocks = sampler.stop()
    ctx.sync()
    lens_h = outd.cpu().numpy().copy()
    outd.zero_()
    tot_doff = timed_calls(lambda: ctx.batch_dev(dxs, dxo, dys, dyo, len(pairs), outd, stream=stream), stream,
                           min(min_s, 0.3), flush=lambda: flush_l2(flush))
    ctx.sync()
    assert np.array_equal(outd.cpu().numpy(), lens_h), "the two batch entry points disagree"
    dof_ms = max_over_ranks(float(np.median(tot_doff)), dist, dev)
    # stage split with the context's stage events (direct launches)
    ctx.set_profiling(True)
    kern, prep = [], []
    for _ in range(7):
        with torch.cuda.stream(stream):
            flush_l2(flush)
        ctx.batch_dev(dxs, dxo, dys, dyo, len(pairs), outd, stream=stream)
        p = ctx.last_profile()
        kern.append(p["fill_ms"])
        prep.append(p["prep_ms"])
    ctx.set_profiling(False)
    lens = outd.cpu().numpy()
    # host-buffer end to end (concatenated pinned host buffers and offsets, as a caller holds them)
    xs_h = torch.from_numpy(xs).pin_memory().numpy()
    ys_h = torch.from_numpy(ys).pin_memory().numpy()
    e2e = host_calls(lambda: ctx.batch_concat(xs_h, xo, ys_h, yo), min_s=0.5)
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
    ctx.close()
    # the serial oracle on a sample of the pairs (and their lengths checked on the way)
    cpu = None
    if rank == 0 and not args.no_cpu:
        oracle.build()
        osample = list(range(0, len(pairs), max(1, len(pairs) // 300)))
        t0 = time.perf_counter()
        want = [oracle.lcs_length(pairs[i][0], pairs[i][1]) for i in osample]
        dt = time.perf_counter() - t0
        ocells = sum(len(pairs[i][0]) * len(pairs[i][1]) for i in osample)
        cpu = {"value": ocells / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
               "sample": f"LCS-length of {len(osample)} of the pairs, one after the other ({ocells:.3g} cells, "
                         f"{dt:.2f} s)",
               "lengths_equal_to_batch": bool(all(int(lens[i]) == w for i, w in zip(osample, want)))}
    t_ms = max_over_ranks(float(np.median(tot)), dist, dev)
    k_ms = max_over_ranks(float(np.median(kern)), dist, dev)
    e2e_s = max_over_ranks(float(np.median(e2e)), dist, dev)
    return {
        "workload": "batch: 10000 pairs, m and n log-uniform in [64, 4096], sigma 4 (half) and 20 (half), lengths only",
        "value": total_cells / (t_ms * 1e-3) / 1e9, "unit": "GCUPS", "ms_per_call": t_ms, "calls_timed": len(tot),
        "timed_s": float(np.sum(tot)) * 1e-3, "cells": total_cells, "pairs": len(all_pairs),
        "parallelism": f"pairs split over {ws} ranks, cells balanced" if ws > 1 else "1 GPU",
        "l2": "explicit 256 MiB L2 flush before every timed call (outside the events)",
        "api": "lcs_batch_dev_hoff (strings and lengths in device memory, offsets in host memory)",
        "device_offsets": {"api": "lcs_batch_dev (offsets in device memory: copied back, stream waited on, then "
                                  "planned)", "ms_per_call": dof_ms,
                           "value": total_cells / (dof_ms * 1e-3) / 1e9, "calls_timed": len(tot_doff)},
        "batch_config": tuned or None,
        "stages_ms": {"prep": float(np.median(prep)), "batch_kernel": k_ms},
        "kernel_gcups": total_cells / (k_ms * 1e-3) / 1e9,
        "roofline": alu_line(total_cells // ws, 5, k_ms, clocks, "k_batch_main", probes, "row_update"),
        "sequential_per_pair": {"gcups": seq_cells / seq_s / 1e9, "pairs_timed": len(sample),
                                "speedup_of_batch": (total_cells / ws / (t_ms * 1e-3)) / (seq_cells / seq_s),
                                "note": "lcs_length_dev per pair, back to back, same GPU"},
        "e2e": {"value": total_cells / e2e_s / 1e9, "unit": "GCUPS", "stat": "median of the timed calls",
                "calls": len(e2e), "h2d_bytes_per_step": int(xs.nbytes + ys.nbytes),
                "d2h_bytes_per_step": 8 * len(pairs),
                "transfer": "lcs_batch on page-locked host buffers: the kernels read the strings in place over the "
                            "host link (no copy into device buffers first), the lengths come back by one copy"},
        "cpu_baseline": cpu,
        "gpu_launches": 3 * len(tot), "clocks": clocks,  # k_batch_prep, k_batch_main, k_batch_combine per call
    }


def run_batch_workload(args):
    """The batch as its own line; under torchrun the batch is split over the ranks by pair (no data exchanged) and
    value = all cells / the slowest rank's time."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    probes = measure_probes(local)
    r = measure_batch(args, dev, probes, ws=ws, rank=rank, dist=dist)
    line = {
        "metric": METRIC, "value": r["value"], "unit": "GCUPS", "n_gpus": ws, "steps": r["calls_timed"],
        "warmup": args.warmup, "ms_per_step": r["ms_per_call"], "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": r["workload"], "cells": r["cells"], "pairs": r["pairs"], "parallelism": r["parallelism"],
                   "l2": r["l2"]},
        **{k: r[k] for k in ("api", "device_offsets", "batch_config", "stages_ms", "kernel_gcups", "roofline",
                              "sequential_per_pair", "e2e", "cpu_baseline", "gpu_launches", "clocks")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---- serving --------------------------------------------------------------------------------------------------------

SERVE_CLASSES = ("short", "long", "traceback")


def serve_class(r: dict) -> str:
    """The server's routing of a request: tracebacks and long length-only pairs to the single-pair workers, short
    length-only pairs (shorter side <= 4096, longer side <= 16384, m*n < 2^24) to the batch workers."""
    m, n = len(r["x"]), len(r["y"])
    if r["traceback"]:
        return "traceback"
    return "short" if min(m, n) <= 4096 and max(m, n) <= 16384 and m * n < (1 << 24) else "long"


def measure_serve(args, dev) -> dict:
    """Poisson request streams at swept rates (m and n log-uniform in [32, 65536], alphabet 4, 20 or 256, 20%
    traceback) through the server: latency from submit to result (measured by the server), p50/p99 and served GCUPS
    per rate; each rate offers at least one second of requests (2000 to 20000). Beside them the per-pair baseline:
    the same request mix run one request at a time through lcs_length / lcs_traceback."""
    from paper_1306_4627_gb300 import gen, lcs
    ctx = lcs.Context(dev.index)
    rates = [float(r) for r in args.rates.split(",")]
    out_rates = []
    sampler = ClockSampler(dev.index).start()
    for rate in rates:
        count = int(min(args.serve_max, max(args.serve_min, rate * args.serve_s)))
        reqs = gen.serve_requests(rate=rate, count=count, seed=gen.BASE_SEED + 4)
        cells = sum(len(r["x"]) * len(r["y"]) for r in reqs)
        srv = lcs.Server(ctx, pair_workers=args.pair_workers)
        for r in reqs[:8]:  # warm the workers' buffers with a few requests
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
        cls = np.array([serve_class(r) for r in reqs])
        out_rates.append({"rate_per_s": rate, "requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                          "p99_ms": float(np.percentile(lat, 99) * 1e3), "gcups": cells / wall / 1e9,
                          "offered_gcups": cells / (reqs[-1]["t"] - reqs[0]["t"]) / 1e9, "wall_s": wall,
                          "by_class": {c: {"requests": int((cls == c).sum()),
                                           "p50_ms": float(np.percentile(lat[cls == c], 50) * 1e3),
                                           "p99_ms": float(np.percentile(lat[cls == c], 99) * 1e3)}
                                       for c in SERVE_CLASSES if (cls == c).any()}})
        print(json.dumps({"serve_rate": out_rates[-1]}), file=sys.stderr, flush=True)
        del reqs
    clocks = sampler.stop()
    # per-pair baseline: the same request mix, one call at a time (service time of each)
    reqs = gen.serve_requests(rate=1000.0, count=min(args.serve_min, 1000), seed=gen.BASE_SEED + 4)
    svc = []
    for r in reqs:
        t1 = time.perf_counter()
        (ctx.traceback if r["traceback"] else ctx.length)(r["x"], r["y"])
        svc.append(time.perf_counter() - t1)
    svc = np.array(svc)
    ctx.close()
    cls = np.array([serve_class(r) for r in reqs])
    best = max(out_rates, key=lambda d: d["gcups"])
    return {
        "workload": "serving: Poisson arrivals, m,n log-uniform [32, 65536], sigma 4/20/256, 20% traceback",
        "value": best["gcups"], "unit": "GCUPS", "rates": out_rates,
        "pair_workers": args.pair_workers or 16,
        "per_pair_baseline": {"p50_ms": float(np.percentile(svc, 50) * 1e3),
                              "p99_ms": float(np.percentile(svc, 99) * 1e3),
                              "gcups": sum(len(r["x"]) * len(r["y"]) for r in reqs) / svc.sum() / 1e9,
                              "requests": len(reqs),
                              "by_class": {c: {"requests": int((cls == c).sum()),
                                               "p50_ms": float(np.percentile(svc[cls == c], 50) * 1e3),
                                               "p99_ms": float(np.percentile(svc[cls == c], 99) * 1e3)}
                                           for c in SERVE_CLASSES if (cls == c).any()},
                              "note": "each request alone through lcs_length / lcs_traceback, one at a time"},
        "classes": "short: length only, shorter side <= 4096, longer side <= 16384 and m*n < 2^24 (batched); long: "
                   "other length-only requests; traceback: every request with traceback",
        "clocks": clocks,
    }


def run_serve_workload(args):
    import torch
    dev = torch.device("cuda", 0)
    r = measure_serve(args, dev)
    best = max(r["rates"], key=lambda d: d["gcups"])
    line = {
        "metric": METRIC, "value": r["value"], "unit": "GCUPS", "n_gpus": 1, "steps": len(r["rates"]),
        "warmup": 1, "ms_per_step": best["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": r["workload"], "pair_workers": r["pair_workers"]},
        "rates": r["rates"], "per_pair_baseline": r["per_pair_baseline"], "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


# ---- the paper's Table 1 shapes -------------------------------------------------------------------------------------

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
    ap.add_argument("--workload", default="all", choices=["all", "pair", "batch", "long", "serve", "table1"],
                    help="all: the 65536^2 traceback step plus every other configuration (default); pair: the "
                         "65536^2 step alone; batch: 10000 pairs; long: 262144^2 length; serve: Poisson request "
                         "streams; table1: the shapes of the paper's Table 1")
    ap.add_argument("--sustain-s", type=float, default=1.0,
                    help="seconds of the headline step timed after the K steps (0 = none)")
    ap.add_argument("--seq-sample", type=int, default=400, help="pairs timed as sequential single-pair launches")
    ap.add_argument("--rates", default="1000,3000,10000,30000,100000", help="serving: request rates per second")
    ap.add_argument("--serve-s", type=float, default=1.0, help="serving: seconds of requests offered per rate")
    ap.add_argument("--serve-min", type=int, default=2000, help="serving: fewest requests per rate")
    ap.add_argument("--serve-max", type=int, default=20000, help="serving: most requests per rate")
    ap.add_argument("--pair-workers", type=int, default=0, help="serving: single-pair workers (0 = the default)")
    ap.add_argument("--variant", default="uniform", choices=["uniform", "mutated"],
                    help="pair workload: independent uniform DNA (default) or Y a mutated copy of X")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    M, N = args.m, args.n
    if (M, N) != (65536, 65536) or args.variant != "uniform":
        args.workload = "pair" if args.workload == "all" else args.workload  # a smaller or other case: that alone
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
