#!/usr/bin/env python3
"""Throughput of the GB300 tridiagonal partition solver.

Default workload: one system of N = 2^26 unknowns, binary64 storage, the
benchmark distribution (b ~ U[4,8], a, c ~ U[-1,1], x* ~ U[-1,1], d = A x*).
A timed step is one solve of that system to binary64 accuracy with inputs
resident in HBM (2 GiB, larger than L2): the headline is the binary32 solve
with one binary64 refinement step (the windowed single pass; error about
1e-13 against x*), and the plain binary64 solve (predictor lookup, Stage 1,
the recursive interface solve, Stage 3) is timed the same way under "fp64".
The same run also times binary32 storage, the plain one-thread-per-system GPU
Thomas baseline, the 4096-system batched workload, the adjoint workload and
the implicit heat step, and reports them under "variants".

Prints ONE JSON line (rank 0).  Under torchrun every rank solves its own
replica (independent problems, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_MAIN = 1 << 26
METRIC = "unknowns solved/sec (N=2^26 to binary64 accuracy: FP32 solve + FP64 refinement; FP64 solve beside it)"
WORKLOAD = "single tridiagonal system N=2^26, binary64 storage, b~U[4,8], a,c~U[-1,1], d=A x*"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# binary64 pipe: 2 operations (FMA or MUL) per clock per SM, the nominal
# 1.25 TFLOP/s over 152 SMs at 2.07 GHz with 2 flops per FMA; the roofline
# uses the rate measured in the same run (tdp_fp64_fma_rate) when it can
FP64_PEAK_GOPS = 152 * 2.07e9 * 2 / 1e9
FP64_PEAK_TFLOPS = FP64_PEAK_GOPS * 2 / 1e3


def stage1_f64_ops(s):
    """Binary64 FMAs and MULs of Stage 1 with kept coefficients per full block
    of s rows: row 1 (reciprocal: 3 FMA; gamma, delta, alpha: 3 MUL), rows
    2..s-1 (pivot, 3 in the reciprocal, delta: 5 FMA; q, gamma, d r, alpha:
    4 MUL), the backward sweep over rows s-3..1 (ap, dp: 2 FMA; gp: 1 MUL)
    and the top interface row (2 FMA, 1 MUL)."""
    fma = 3 + 5 * (s - 2) + 2 * (s - 3) + 2
    mul = 3 + 4 * (s - 2) + (s - 3) + 1
    return fma, mul


def stage1_f64_roofline(ms, n, s, hbm_peak_gbs, traffic=None, peak_gops=None, peak_source=None):
    """ALU roofline of the binary64 Stage 1 from its event-timed launch (ms):
    binary64 pipe operations per second against the pipe's rate (measured in
    this run when given, else the derived 2 per clock per SM), and the same
    work in flops against the FMA-only flop peak."""
    fma, mul = stage1_f64_ops(s)
    ops = (fma + mul) * n / s
    flops = (2 * fma + mul) * n / s
    gops = ops / (ms * 1e-3) / 1e9
    tflops = flops / (ms * 1e-3) / 1e12
    peak = peak_gops or FP64_PEAK_GOPS
    return {"bound": "alu", "kernel": "stage1_keep_f64", "achieved": gops, "peak": peak,
            "unit": "Gop/s", "frac": gops / peak, "traffic": traffic,
            "peak_source": peak_source or "derived: 152 SMs x 2.07 GHz x 2 binary64 FMA or MUL per clock",
            "peak_derived": FP64_PEAK_GOPS, "ops_per_row": (fma + mul) / s, "fma_mul_per_block": [fma, mul],
            "achieved_tflops": tflops, "peak_tflops": 2 * peak / 1e3, "frac_flops": tflops / (2 * peak / 1e3),
            "algorithmic_bytes_per_row": 56 + 64 / s,
            "hbm_frac_of_kernel": (56 + 64 / s) * n / (ms * 1e-3) / 1e9 / hbm_peak_gbs}


def window_geometry(tdp):
    """(rows per thread, halo rows, owned rows per tile) of the windowed pass."""
    sw = tdp.tdp_get_tuning(tdp.TUNE_WINDOW_SW)
    halo = max(16, min(tdp.tdp_get_tuning(tdp.TUNE_WINDOW_HALO), 64)) & ~3
    return sw, halo, 256 * sw - 2 * halo


def window_roofline(tdp, ms, n, iters, hbm_peak_gbs, fp64_peak_gops, traffic=None):
    """HBM roofline of the windowed pass (k_window<double>) from its
    event-timed launch: 32 bytes read and 8 written per row (algorithmic),
    against the measured copy bandwidth; beside it the binary64 pipe: per
    correction 3 FMA per window row (the residual) and 1 add per owned row
    (the update)."""
    sw, halo, tr = window_geometry(tdp)
    gbs = 40 * n / (ms * 1e-3) / 1e9
    ops_row = iters * (3 * (256 * sw) / tr + 1)
    gops = ops_row * n / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "window_refine", "achieved": gbs, "peak": hbm_peak_gbs, "unit": "GB/s",
            "frac": gbs / hbm_peak_gbs, "traffic": traffic, "algorithmic_bytes_per_row": 40,
            "geometry": {"rows_per_thread": sw, "halo": halo, "tile_rows": tr, "window_rows": 256 * sw},
            "fp64_ops_per_row": ops_row, "fp64_achieved_gops": gops, "fp64_peak_gops": fp64_peak_gops,
            "fp64_frac": gops / fp64_peak_gops}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def batched_s(tdp, Sb, code):
    """The sub-system size tdp_solve_batched(s=0) uses: batches of systems of
    at least 4096 rows on average run as one block-diagonal system with the
    single-system model's s (if that s suits the 16-byte tiles), others
    with the model at the mean system size."""
    if tdp.tdp_get_tuning(tdp.TUNE_BATCH_FLAT) and Sb.batch >= 2 and Sb.n >= 4096 * Sb.batch:
        s1 = tdp.tdp_predict_s(Sb.n, 1, code)
        if code == tdp.F32_REFINE or s1 % (2 if code == tdp.F64 else 4) == 0:
            return s1
    return tdp.tdp_predict_s(max(1, Sb.n // Sb.batch), Sb.batch, code)


def measured_traffic(kernel, s, n):
    """DRAM bytes per launch of ``kernel`` from the committed ncu capture
    (profiles/traffic.json), scaled to n rows; None when the kernel sources
    changed since the capture or the sub-system size differs."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    except (OSError, KeyError, ValueError):
        return None
    if h.hexdigest() != rec["sha256"] or int(rec["s"]) != int(s):
        return None
    return rec["bytes_per_row"] * n


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def weak_value(n_per_rank, world, ms_max):
    """Whole-job unknowns/s: every rank solved its own n_per_rank unknowns in
    at most ms_max milliseconds."""
    return world * n_per_rank / (ms_max * 1e-3)


def run_reference_guard(rank, fn):
    """The reference arm runs on rank 0 only; the other ranks return at once."""
    if rank == 0:
        fn()


def barrier_max(value, world, device):
    """Barrier, then the maximum of ``value`` over ranks."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------
def run_reference(args, world, rank):
    run_reference_guard(rank, lambda: _reference_line(args))


def _reference_line(args):
    import oracle

    S = W.single(N_MAIN, seed=0)
    # bounded sample: the whole system when the run stays within ~2 minutes
    t0 = time.perf_counter()
    oracle.thomas(S.a, S.b, S.c, S.d)
    t_one = time.perf_counter() - t0
    n_sample = N_MAIN if t_one * (args.steps + args.warmup) < 120 else max(1 << 20, int(N_MAIN * 120 / (
        t_one * (args.steps + args.warmup))))
    sl = slice(0, n_sample)
    a, b, c, d = (np.ascontiguousarray(v[sl]) for v in (S.a, S.b, S.c, S.d))
    for _ in range(args.warmup):
        oracle.thomas(a, b, c, d)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.thomas(a, b, c, d)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_sample * args.steps / total
    sample = f"oracle Thomas (binary64, one core) on the first {n_sample} rows of the N=2^26 system per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_MAIN, "batch": 1},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_info()[0], "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def cuda_time_flushed(fn, steps, warmup, stream, flush):
    """Median milliseconds of ``steps`` calls, L2 flushed before each one by
    writing ``flush`` (a device buffer larger than L2) on ``stream``; only the
    call itself is inside its pair of CUDA events."""
    import torch

    for _ in range(warmup):
        fn()
    times = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def cuda_time_each(fn, steps, warmup, stream):
    """(median, mean) milliseconds of ``steps`` calls, each between its own
    pair of CUDA events on ``stream``.  The median: the host link of a shared
    box has episodes two to three times slower that hit any copy (copies of
    the same bytes alone included), and one of them would dominate a mean."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times), statistics.fmean(times)


def cuda_time(fn, steps, warmup, stream):
    """Milliseconds per call over ``steps`` calls (CUDA events on ``stream``)."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def profile_kernels(tdp, fn, steps):
    """{kernel: (launches, mean ms)} for ``steps`` calls (library event timing)."""
    import torch

    torch.cuda.synchronize()
    tdp.tdp_profile_enable(True)
    for _ in range(steps):
        fn()
    torch.cuda.synchronize()
    prof = tdp.tdp_profile_summary()
    tdp.tdp_profile_enable(False)
    return {k: (v[0], v[1] / max(1, v[0])) for k, v in prof.items()}


def run_ours(args, world, rank, local):
    import torch

    import paper_2510_27351_gb300 as tdp

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)
    stream = torch.cuda.current_stream()
    pk, pk_src = peaks()
    hbm_peak = float(pk.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))

    # ---- inputs of the main workload (host, pinned copies for e2e) ----
    t0 = time.time()
    S = W.single(N_MAIN, seed=rank)
    log(f"[bench] generated N=2^26 in {time.time() - t0:.1f}s")
    host = {k: torch.from_numpy(getattr(S, k)).pin_memory() for k in ("a", "b", "c", "d")}
    dev = {k: v.to(device, non_blocking=True) for k, v in host.items()}
    x = torch.empty(N_MAIN, dtype=torch.float64, device=device)
    torch.cuda.synchronize()
    s_main = tdp.tdp_predict_s(N_MAIN, 1, tdp.F64)
    fp64_rate, fp64_ms = tdp.tdp_fp64_fma_rate(stream)
    fp64_peak = fp64_rate / 1e9
    fp64_src = f"measured in this run: tdp_fp64_fma_rate, {fp64_rate:.4g} binary64 FMA/s ({fp64_ms:.2f} ms launch)"

    def step_f64():
        s = tdp.tdp_predict_s(N_MAIN, 1, tdp.F64)
        tdp.tdp_solve(dev["a"], dev["b"], dev["c"], dev["d"], x, N_MAIN, s, tdp.F64, 0, stream)

    def step_refine():
        tdp.tdp_solve(dev["a"], dev["b"], dev["c"], dev["d"], x, N_MAIN, 0, tdp.F32_REFINE, 1, stream)

    def check(step):
        """Error against x* of the timed configuration, and the status bits
        (a set fallback bit would mean the exact solve answered instead)."""
        tdp.tdp_set_checked(True)
        step()
        bits = int(tdp.LIB.tdp_last_status_bits())
        tdp.tdp_set_checked(False)
        torch.cuda.synchronize()
        return float((x.cpu().numpy() - S.xstar).__abs__().max() / np.abs(S.xstar).max()), bits

    def timed(step):
        """ms per step over args.steps steps after args.warmup, the max over
        ranks, with the clocks sampled during the load and our launches counted."""
        with ClockSampler(local) as clk:
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            barrier_max(0.0, world, device)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            la = tdp.tdp_launch_count()
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            lb = tdp.tdp_launch_count()
            ms_ = e0.elapsed_time(e1) / args.steps
            # keep the same load (untimed) for a moment so that the clock
            # samples cover at least half a second of it
            t_end = time.time() + 0.6
            while time.time() < t_end:
                for _ in range(20):
                    step()
                torch.cuda.synchronize()
        return barrier_max(ms_, world, device), clk.summary(), lb - la

    # ---- headline: binary32 solve + one binary64 correction (windowed pass) ----
    err_refine, bits_refine = check(step_refine)
    ms, clocks, gpu_launches = timed(step_refine)
    value = weak_value(N_MAIN, world, ms)
    prof = profile_kernels(tdp, step_refine, max(3, min(args.steps, 10)))
    dom = max(prof.items(), key=lambda kv: kv[1][0] * kv[1][1])  # largest total time per step
    win = prof.get("window_refine")
    roof = None
    if win:
        roof = window_roofline(tdp, win[1], N_MAIN, 1, hbm_peak, fp64_peak,
                               measured_traffic("window_refine", window_geometry(tdp)[0], N_MAIN))
    solve_hbm_frac = value / world * 40 / 1e9 / hbm_peak

    # ---- the binary64 solve of the same system ----
    err_xstar, _ = check(step_f64)
    ms64, clocks64, launches64 = timed(step_f64)
    prof64 = profile_kernels(tdp, step_f64, max(3, min(args.steps, 10)))
    st1 = prof64.get("stage1_keep_f64")
    roof64 = None
    if st1:
        roof64 = stage1_f64_roofline(st1[1], N_MAIN, s_main, hbm_peak,
                                     measured_traffic("stage1_keep_f64", s_main, N_MAIN), fp64_peak, fp64_src)
    fp64 = {"value": weak_value(N_MAIN, world, ms64), "unit": "unknowns/s", "ms_per_step": ms64, "s": s_main,
            "hbm_frac_40B": weak_value(N_MAIN, world, ms64) / world * 40 / 1e9 / hbm_peak,
            "rel_err_vs_xstar": err_xstar, "roofline": roof64, "kernels_ms": {k: v[1] for k, v in prof64.items()},
            "gpu_launches": launches64, "clocks": clocks64}

    # ---- end to end through the public API with host buffers ----
    host_x = torch.empty(N_MAIN, dtype=torch.float64).pin_memory()

    def step_e2e():
        # the library's host-array entry: the windowed pass streamed by chunks,
        # copies in and out overlapping the solve
        tdp.tdp_solve_host(host["a"], host["b"], host["c"], host["d"], host_x, N_MAIN, 0, tdp.F32_REFINE, 1, stream)

    def step_e2e64():
        # binary64: the copies pipelined with Stage 1 and Stage 3
        tdp.tdp_solve_host(host["a"], host["b"], host["c"], host["d"], host_x, N_MAIN, s_main, tdp.F64, 0, stream)

    e2e_ms, e2e_mean = cuda_time_each(step_e2e, max(5, args.steps // 2), 2, stream)
    e2e64_ms, e2e64_mean = cuda_time_each(step_e2e64, max(5, args.steps // 2), 2, stream)
    e2e_ms = barrier_max(e2e_ms, world, device)
    e2e64_ms = barrier_max(e2e64_ms, world, device)
    e2e = {"value": world * N_MAIN / (e2e_ms * 1e-3), "unit": "unknowns/s", "h2d_bytes_per_step": 4 * 8 * N_MAIN,
           "d2h_bytes_per_step": 8 * N_MAIN, "ms_per_step": e2e_ms, "ms_mean": e2e_mean, "statistic": "median",
           "fp64": {"value": world * N_MAIN / (e2e64_ms * 1e-3), "ms_per_step": e2e64_ms, "ms_mean": e2e64_mean}}

    variants = {}
    if not args.main_only:
        variants = run_variants(args, tdp, S, dev, x, stream, hbm_peak, device)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(S, W.batched(4096, 64, 65536, seed=0))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_MAIN, "batch": 1, "refine_iters": 1,
                       "parallelism": f"replicas{world}", "l2": "inputs (2 GiB) larger than L2; no flush"},
            "roofline": roof, "hbm_frac_of_whole_solve": solve_hbm_frac, "peaks_source": pk_src,
            "hbm_peak_gbs": hbm_peak, "fp64_peak": {"gops": fp64_peak, "source": fp64_src},
            "kernels_ms": {k: v[1] for k, v in prof.items()}, "dominant_kernel": dom[0],
            "rel_err_vs_xstar": err_refine, "status_bits": bits_refine, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clocks, "fp64": fp64, "cpu_baseline": cpu, "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def cpu_info():
    """(CPU model string, usable host cores) of this machine."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform

    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return model or platform.machine(), cores


def _timed_reps(fn, seconds):
    t_end = time.perf_counter() + seconds
    reps, t = 0, 0.0
    while time.perf_counter() < t_end or reps == 0:
        t0 = time.perf_counter()
        fn()
        t += time.perf_counter() - t0
        reps += 1
    return reps, t


def cpu_baseline(S, Sb=None):
    """The oracle's binary64 Thomas on the host: one core on the whole
    N = 2^26 system, and every host core at once (a thread per core; the
    oracle's C code runs outside the interpreter lock) on equal slices of it
    solved as independent systems (a throughput figure for the same rows, not
    the same solve) and on the systems of the 4096-system batch."""
    import concurrent.futures as cf

    import oracle

    model, cores = cpu_info()
    reps, t = _timed_reps(lambda: oracle.thomas(S.a, S.b, S.c, S.d), 8.0)
    one = {"value": reps * N_MAIN / t, "cores": 1,
           "sample": f"oracle Thomas on the full N=2^26 system, {reps} repetitions (~8 s)"}
    bounds = np.linspace(0, N_MAIN, cores + 1).astype(np.int64)
    slices = [(int(lo), int(hi)) for lo, hi in zip(bounds[:-1], bounds[1:])]
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        def all_slices():
            list(ex.map(lambda r: oracle.thomas(S.a[r[0]:r[1]], S.b[r[0]:r[1]], S.c[r[0]:r[1]], S.d[r[0]:r[1]]),
                        slices))

        reps_m, t_m = _timed_reps(all_slices, 8.0)
        batched = None
        if Sb is not None:
            groups = np.array_split(np.arange(Sb.batch), cores)

            def one_group(g):
                lo, hi = int(Sb.offsets[g[0]]), int(Sb.offsets[g[-1] + 1])
                oracle.thomas_batched(Sb.a[lo:hi], Sb.b[lo:hi], Sb.c[lo:hi], Sb.d[lo:hi],
                                      offsets=Sb.offsets[g[0]:g[-1] + 2] - lo)

            reps_b, t_b = _timed_reps(lambda: list(ex.map(one_group, [g for g in groups if len(g)])), 5.0)
            batched = {"value": reps_b * Sb.n / t_b, "cores": cores,
                       "sample": f"oracle Thomas per system, 4096-system batch (sum N = {Sb.n}), {reps_b} passes"}
    return {"value": reps_m * N_MAIN / t_m, "unit": "unknowns/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle Thomas on {cores} equal slices of the N=2^26 rows, one thread each, "
                      f"{reps_m} passes (~8 s)",
            "cpu_model": model, "nproc": os.cpu_count(), "one_core": one, "batched_4096": batched}


def run_variants(args, tdp, S, dev, x, stream, hbm_peak, device):
    import torch

    out = {}
    steps = max(3, min(args.steps, 10))
    import oracle

    def hbm(ms, bytes_):
        return bytes_ / (ms * 1e-3) / 1e9 / hbm_peak

    # binary32 + binary64 refinement on the same system by the exact three-pass
    # schedule (the windowed pass off): the path the windowed pass falls back on
    # in spirit, and the previous default
    s_r = tdp.tdp_predict_s(N_MAIN, 1, tdp.F32_REFINE)
    tdp.tdp_set_tuning(tdp.TUNE_WINDOW, 0)
    try:
        fn = lambda: tdp.tdp_solve(dev["a"], dev["b"], dev["c"], dev["d"], x, N_MAIN, s_r, tdp.F32_REFINE, 1,
                                   stream)
        ms = cuda_time(fn, steps, 2, stream)
        fn()
        torch.cuda.synchronize()
        err = float(np.abs(x.cpu().numpy() - S.xstar).max() / np.abs(S.xstar).max())
        prof = profile_kernels(tdp, fn, 3)
    finally:
        tdp.tdp_set_tuning(tdp.TUNE_WINDOW, 1)
    out["fp32_refine1_three_pass"] = {"ms": ms, "unknowns_per_s": N_MAIN / (ms * 1e-3),
                                      "hbm_frac_40B": hbm(ms, 40 * N_MAIN), "s": s_r, "rel_err_vs_xstar": err,
                                      "kernels_ms": {k: v[1] for k, v in prof.items()}}
    # binary32 storage
    s_f = tdp.tdp_predict_s(N_MAIN, 1, tdp.F32)
    d32 = {k: v.float() for k, v in dev.items()}
    x32 = torch.empty(N_MAIN, dtype=torch.float32, device=device)
    fn = lambda: tdp.tdp_solve(d32["a"], d32["b"], d32["c"], d32["d"], x32, N_MAIN, s_f, tdp.F32, 0, stream)
    ms = cuda_time(fn, steps, 2, stream)
    err = float(np.abs(x32.double().cpu().numpy() - S.xstar).max() / np.abs(S.xstar).max())
    prof = profile_kernels(tdp, fn, 3)
    out["fp32"] = {"ms": ms, "unknowns_per_s": N_MAIN / (ms * 1e-3), "hbm_frac_20B": hbm(ms, 20 * N_MAIN), "s": s_f,
                   "rel_err_vs_xstar": err, "kernels_ms": {k: v[1] for k, v in prof.items()}}
    del d32, x32
    # plain GPU Thomas, one thread per system: rate measured on the first 2^16 rows
    nt = 1 << 16
    off = torch.tensor([0, nt], dtype=torch.int64, device=device)
    sl = {k: v[:nt].contiguous() for k, v in dev.items()}
    xt = torch.empty(nt, dtype=torch.float64, device=device)
    fn = lambda: tdp.tdp_thomas_batched(off, 1, nt, sl["a"], sl["b"], sl["c"], sl["d"], xt, tdp.F64, stream)
    ms = cuda_time(fn, 2, 1, stream)
    out["thomas_gpu_single"] = {"ms_for_2^16_rows": ms, "unknowns_per_s": nt / (ms * 1e-3),
                                "note": "one GPU thread runs sequential Thomas; rate independent of N"}
    del sl, xt
    # the small single system N = 65536 (fits in L2: latency-bound): per solve,
    # launched on the stream and replayed from a CUDA graph
    Sl = W.single(1 << 16, seed=0)
    ld = {k: torch.from_numpy(getattr(Sl, k)).to(device) for k in ("a", "b", "c", "d")}
    lx = torch.empty(1 << 16, dtype=torch.float64, device=device)
    lat = {}
    for name, code, s_l, it in (("fp64_s32", tdp.F64, 32, 0), ("fp32_refine1", tdp.F32_REFINE, 0, 1)):
        call = lambda st, code=code, s_l=s_l, it=it: tdp.tdp_solve(ld["a"], ld["b"], ld["c"], ld["d"], lx, 1 << 16,
                                                                    s_l, code, it, st)
        ms = cuda_time(lambda: call(stream), 50, 5, stream)
        g = tdp.CapturedSolve(call)
        ms_graph = cuda_time(g.replay, 50, 5, torch.cuda.current_stream())
        del g
        torch.cuda.synchronize()
        err = float(np.abs(lx.cpu().numpy() - Sl.xstar).max() / np.abs(Sl.xstar).max())
        lat[name] = {"us": 1e3 * ms, "us_graph": 1e3 * ms_graph, "unknowns_per_s_graph": (1 << 16) / (ms_graph * 1e-3),
                     "rel_err_vs_xstar": err}
    out["latency_65536"] = lat
    del ld, lx
    # batched: 4096 systems, N log-uniform in [64, 65536]
    Sb = W.batched(4096, 64, 65536, seed=0)
    bdev = {k: torch.from_numpy(getattr(Sb, k)).to(device) for k in ("a", "b", "c", "d")}
    boff = torch.from_numpy(Sb.offsets).to(device)
    bx = torch.empty(Sb.n, dtype=torch.float64, device=device)
    res = {"total_n": Sb.n}
    for name, code, it in (("fp64", tdp.F64, 0), ("fp32_refine1", tdp.F32_REFINE, 1)):
        fn = lambda: tdp.tdp_solve_batched(boff, Sb.batch, Sb.n, bdev["a"], bdev["b"], bdev["c"], bdev["d"], bx, 0,
                                           code, it, stream)
        ms = cuda_time(fn, steps, 2, stream)
        err = float((bx.cpu().numpy() - Sb.xstar).__abs__().max() / np.abs(Sb.xstar).max())
        # the same solve captured once into a CUDA graph and replayed
        g = tdp.CapturedSolve(lambda st: tdp.tdp_solve_batched(boff, Sb.batch, Sb.n, bdev["a"], bdev["b"],
                                                                bdev["c"], bdev["d"], bx, 0, code, it, st))
        ms_graph = cuda_time(g.replay, steps, 2, torch.cuda.current_stream())  # replay() launches there
        res[name] = {"ms": ms, "ms_graph": ms_graph, "unknowns_per_s": Sb.n / (ms * 1e-3),
                     "unknowns_per_s_graph": Sb.n / (ms_graph * 1e-3), "hbm_frac_40B": hbm(ms, 40 * Sb.n),
                     "s": batched_s(tdp, Sb, code), "rel_err_vs_xstar": err}
        del g
    fn = lambda: tdp.tdp_thomas_batched(boff, Sb.batch, Sb.n, bdev["a"], bdev["b"], bdev["c"], bdev["d"], bx,
                                        tdp.F64, stream)
    ms = cuda_time(fn, 2, 1, stream)
    res["thomas_gpu"] = {"ms": ms, "unknowns_per_s": Sb.n / (ms * 1e-3)}
    out["batched_4096"] = res
    del bdev, bx
    # adjoint: 1024 systems of 8192, loss weights w ~ N(0,1)
    Sa = W.uniform_batch(1024, 8192, seed=0)
    adev = {k: torch.from_numpy(getattr(Sa, k)).to(device) for k in ("a", "b", "c", "d")}
    aoff = torch.from_numpy(Sa.offsets).to(device)
    ax = torch.empty(Sa.n, dtype=torch.float64, device=device)
    tdp.tdp_solve_batched(aoff, Sa.batch, Sa.n, adev["a"], adev["b"], adev["c"], adev["d"], ax, 0, tdp.F64, 0,
                          stream)
    g = torch.from_numpy(W.loss_weights(Sa.n, seed=0)).to(device)
    grads = [torch.empty_like(ax) for _ in range(4)]
    res = {}
    for name, code in (("fp64", tdp.F64), ("fp32_refine1", tdp.F32_REFINE)):
        fn = lambda: tdp.tdp_solve_backward(aoff, Sa.batch, Sa.n, adev["a"], adev["b"], adev["c"], ax, g, *grads, 0,
                                            code, stream)
        ms = cuda_time(fn, steps, 2, stream)
        res[name] = {"ms": ms, "unknowns_per_s": Sa.n / (ms * 1e-3), "hbm_frac_72B": hbm(ms, 72 * Sa.n)}
    out["adjoint_1024x8192"] = res
    del adev, ax, grads
    # many right-hand sides of one matrix: 16 columns of a 2^22-row system,
    # one factorisation, against the same columns as 16 separate solves
    nm, km = 1 << 22, 16
    Sm = W.single(nm, seed=3)
    mdev = {k: torch.from_numpy(getattr(Sm, k)).to(device) for k in ("a", "b", "c")}
    Dm = torch.from_numpy(W.rhs_columns(nm, km, seed=3).reshape(-1)).to(device)
    Xm = torch.empty_like(Dm)
    fn = lambda: tdp.tdp_solve_multi(mdev["a"], mdev["b"], mdev["c"], Dm, Xm, nm, km, nm, nm, 0, tdp.F64, stream)
    ms = cuda_time(fn, steps, 2, stream)

    def separate():
        for j in range(km):
            tdp.tdp_solve(mdev["a"], mdev["b"], mdev["c"], Dm[j * nm:(j + 1) * nm], Xm[j * nm:(j + 1) * nm], nm, 0,
                          tdp.F64, 0, stream)

    ms_sep = cuda_time(separate, max(3, steps // 4), 1, stream)
    out["multi_rhs_2^22x16"] = {"ms": ms, "unknowns_per_s": km * nm / (ms * 1e-3), "separate_solves_ms": ms_sep,
                                "s": min(64, max(16, 4 * tdp.tdp_predict_s(nm, 1, tdp.F64))), "dtype": "f64"}
    del mdev, Dm, Xm
    # implicit heat step on 2048^2: row sweep then column sweep
    H = W.heat(2048, 0.5, seed=0)
    hd = {k: torch.from_numpy(np.ascontiguousarray(getattr(H, k)).reshape(-1)).to(device) for k in ("a", "b", "c", "u")}
    r1 = torch.empty_like(hd["u"])
    r2 = torch.empty_like(hd["u"])

    def heat():
        tdp.tdp_solve_strided(2048, 2048, 2048, 1, hd["a"], hd["b"], hd["c"], hd["u"], r1, 0, tdp.F32_REFINE, 1,
                              stream)
        tdp.tdp_solve_strided(2048, 2048, 1, 2048, hd["a"], hd["b"], hd["c"], r1, r2, 0, tdp.F32_REFINE, 1, stream)

    # the step's arrays (32 MiB each) fit in L2: flush it before every repetition
    flush = torch.empty(64 << 20, dtype=torch.float32, device=device)
    ms = cuda_time_flushed(heat, steps, 2, stream, flush)
    out["heat_2048"] = {"ms": ms, "unknowns_per_s": 2 * 2048 * 2048 / (ms * 1e-3), "dtype": "fp32_refine1",
                        "l2": "flushed before each repetition (256 MiB write)"}

    # the same step through the constant-coefficient path (d in, x out), with s
    # from the constant-path autotuner; binary64 storage runs binary64
    # arithmetic there for TDP_F32_REFINE too
    from paper_2510_27351_gb300 import tune

    def step(s):
        tdp.tdp_solve_const(-0.5, 2.0, -0.5, hd["u"], r1, 2048, 2048, 2048, 1, s, tdp.F32_REFINE, 1, stream)
        tdp.tdp_solve_const(-0.5, 2.0, -0.5, r1, r2, 2048, 2048, 1, 2048, s, tdp.F32_REFINE, 1, stream)

    s_best, _ = tune.autotune_const(step)
    fn = lambda: step(s_best)
    ms = cuda_time_flushed(fn, steps, 2, stream, flush)
    out["heat_2048_const"] = {"ms": ms, "unknowns_per_s": 2 * 2048 * 2048 / (ms * 1e-3), "s": s_best,
                              "dtype": "f64 (binary64 storage and arithmetic)",
                              "l2": "flushed before each repetition (256 MiB write)",
                              "kernels_ms": {k: v[1] for k, v in profile_kernels(tdp, fn, 3).items()}}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--main-only", action="store_true", help="skip the variant workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        log("[bench] warmup raised to 3")
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
