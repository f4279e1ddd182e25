"""Benchmark: explicit time marching of the 2D wave equation on one GB300.

Workload (one benchmark step): the 9-point and the 13-point scheme of
arXiv:1904.04048 (Section 6), FP32 storage, 4096 x 4096 periodic grid,
h = 1/4096, c = 1, lambda = 0.9 x each scheme's stability limit, 2000 time
levels each (the first step, Eq. A1, then 1999 two-steps, Eq. A2), followed
by an FP64 norm of the final field copied to the host.  Inputs: 16 seeded
Gaussian pulses for u0 and band-limited random noise for v0 (seed 2019).

Metric: point-updates per second (one point-update = one grid node advanced
one time level), in units of 1e9.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun with one rank per GPU; every rank runs the same
workload on its own GPU (independent replicas, weak scaling) and the value
is the total over ranks divided by the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 4096
STEPS_PER_SCHEME = 2000
SCHEMES = (9, 13)
SEED = 2019
METRIC = "G point-updates/s"
WORKLOAD = ("9-point + 13-point schemes, FP32 storage, 4096^2 periodic grid, lambda = 0.9 lambda_max, "
            "2000 time levels each (first step + 1999 two-steps), 16 Gaussian pulses + band-limited "
            "noise (seed 2019), FP64 norm of the final field to host")

# FP32 operations (add, subtract, multiply or fused multiply-add, one each) of
# one two-step node-update as the schemes are written (Section 6): the class
# sums of Eq. notations2 with their -4 u_ij terms, the products by the
# coefficients, and 2 u^k - u^{k-1} + Lambda.
FP32_OPS = {5: 9, 9: 14, 13: 19}

# Kernel names by WAVE2D_KERNEL_* value (the profiles use the same names).
KNAME = {1: "k2_simple", 2: "k2_tma", 3: "k3_temporal", 4: "k5_stream", 5: "k2_persist"}
KSHORT = {1: "simple", 2: "tma", 3: "temporal", 4: "stream", 5: "persistent"}

# DRAM bytes (read + write) of one launch of a kernel at the benchmark size,
# from an ncu capture of the same kernel source (see the profiles directory),
# keyed by (kernel, hash of that kernel's sources without comments, scheme,
# rows per tile or strip, levels per launch) so that a figure is dropped once
# the kernel or the autotuner's choice changes.
NCU_TRAFFIC = {("k5_stream", "5d1d406f6b836821", 9, 64, 6): 164908032 + 92143616,
               ("k5_stream", "5d1d406f6b836821", 13, 64, 4): 181641216 + 92357888,
               ("k2_tma", "abb92c6c2c27d289", 13, 0, 1): 135369216 + 20198400}

# Sources each kernel is built from (the hash keys of NCU_TRAFFIC).
KERNEL_SOURCES = {"k2_tma": ("kernels.cuh", "stencil_ops.cuh"),
                  "k3_temporal": ("kernels.cuh", "kernels_temporal.cuh", "stencil_ops.cuh"),
                  "k5_stream": ("kernels.cuh", "kernels_stream.cuh", "stencil_ops.cuh")}

# The autotuner's choice on GB300 (kernel, rows per tile or strip, levels
# per launch), used by --fixed-tuning for profiler runs.
FIXED_TUNING = {9: ("stream", 64, 6), 13: ("stream", 64, 4)}


def strip_comments(src: str) -> str:
    """C++ source without comments and blank space: what the compiler sees of
    it up to layout (string literals in these headers hold no comment marks)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash(kernel: str) -> str:
    hsh = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_1904_04048_gb300", "csrc", f), encoding="utf-8") as fh:
            hsh.update(strip_comments(fh.read()).encode())
    return hsh.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = str(device_index)
        try:
            import torch
            self.dev = "GPU-" + str(torch.cuda.get_device_properties(device_index).uuid)
        except Exception:
            pass
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.dev, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ multi-rank
def reduce_max(values, device):
    """Element-wise maximum of per-rank timings over all ranks (every rank
    runs its own replica; the slowest one bounds the whole job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_value(units_per_rank, world, max_elapsed_s, scale=1e9):
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * units_per_rank / max_elapsed_s / scale


# --------------------------------------------------------------- CPU oracle
def time_oracle(u0, v0, budget_s: float):
    """Time the FP64 oracle (as it stands) on a bounded sample of the
    workload: both schemes on the full 4096^2 grid for a few time levels."""
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    h = 1.0 / N
    from initial_data import LAMBDA_MAX
    # probe one level per scheme, then size the sample to the budget
    t0 = time.perf_counter()
    for s in SCHEMES:
        lam = 0.9 * LAMBDA_MAX[s]
        oracle.run(s, u0, v0, lam, lam * h, 1, bc=oracle.BC_PERIODIC)
    probe = time.perf_counter() - t0
    levels = max(2, int(budget_s / max(probe, 1e-3)))
    t0 = time.perf_counter()
    for s in SCHEMES:
        lam = 0.9 * LAMBDA_MAX[s]
        oracle.run(s, u0, v0, lam, lam * h, levels, bc=oracle.BC_PERIODIC)
    dt = time.perf_counter() - t0
    pts = len(SCHEMES) * levels * N * N
    return {"value": pts / dt / 1e9, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"both schemes on the full {N}^2 grid, {levels} time levels each "
                      f"({pts:.3e} point-updates, {dt:.1f} s)"}


def time_oracle_table(u0, v0, budget_s: float = 1.5):
    """The FP64 oracle, as it stands, on one host thread and on all of them,
    over bounded samples of the paper's workloads (each sample sized to about
    budget_s per thread count): the 5-point FP64 256^2 run, the 4096^2
    benchmark grid (both schemes), periodic plane waves at N <= 1024, the
    first instances of the batched workload and the first requests of the
    served stream (each instance run for the same number of levels)."""
    import numpy as np

    import oracle
    from initial_data import (BC_PERIODIC, BC_ZERO, LAMBDA_MAX, batch_instances, gaussian_pulse, instance_ic,
                              plane_wave_ic, plane_wave_k, request_stream)
    cases = {}
    g = gaussian_pulse(256, 256, 1.0 / 256, BC_ZERO, sigma=0.05)
    cases["5point_fp64_256"] = ("5-point, 256^2, lambda 0.5, zero boundary, centred Gaussian",
                                [(5, g, np.zeros_like(g), 0.5, 0.5 / 256, BC_ZERO)])
    cases["benchmark_4096"] = ("9- and 13-point, 4096^2 periodic, the benchmark's inputs",
                               [(s, u0, v0, 0.9 * LAMBDA_MAX[s], 0.9 * LAMBDA_MAX[s] / N, BC_PERIODIC)
                                for s in SCHEMES])
    waves = []
    for n, s, m in ((512, 5, (1, 0)), (1024, 9, (3, 4)), (1024, 13, (32, 16))):
        k1, k2 = plane_wave_k(n, *m)
        pu, pv = plane_wave_ic(n, n, 1.0 / n, k1, k2, BC_PERIODIC)
        lam = 0.9 * LAMBDA_MAX[s]
        waves.append((s, pu, pv, lam, lam / n, BC_PERIODIC))
    cases["plane_waves_le_1024"] = ("periodic plane waves: 5-point 512^2 mode (1,0), 9-point 1024^2 mode (3,4), "
                                    "13-point 1024^2 mode (32,16)", waves)

    def inst_jobs(insts):
        jobs = []
        for i in insts:
            iu, iv, ih = instance_ic(i)
            jobs.append((i.scheme, iu, iv, i.lam, i.lam * ih, BC_ZERO))
        return jobs
    cases["batched_first_16"] = ("the first 16 of the 512 batched instances (seed 4)",
                                 inst_jobs(batch_instances(512, seed=4)[:16]))
    cases["served_first_8"] = ("the first 8 of the 2000 served requests (seed 5)",
                               inst_jobs([r.inst for r in request_stream(2000, seed=5)[:8]]))

    def run_all(jobs, levels):
        for s, a, b, lam, tau, bc in jobs:
            oracle.run(s, a, b, lam, tau, levels, bc=bc)

    all_threads = os.cpu_count() or 1
    out = {}
    for key, (what, jobs) in cases.items():
        row = {"sample": what}
        for threads in (1, all_threads):
            used = oracle.set_threads(threads)
            t0 = time.perf_counter()
            run_all(jobs, 2)
            probe = time.perf_counter() - t0
            levels = max(2, int(2 * budget_s / max(probe, 1e-4)))
            t0 = time.perf_counter()
            run_all(jobs, levels)
            dt = time.perf_counter() - t0
            pts = levels * sum(j[1].size for j in jobs)
            row[f"threads_{used}"] = {"value": round(pts / dt / 1e9, 5), "levels": levels, "seconds": round(dt, 2)}
        out[key] = row
    oracle.set_threads(all_threads)
    return {"unit": "G point-updates/s", "kind": "oracle", "rows": out}


# ----------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from initial_data import BC_PERIODIC, LAMBDA_MAX, pulses_and_noise
    from paper_1904_04048_gb300 import wave2d as w

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w.lib()
    u0, v0 = pulses_and_noise(N, seed=SEED)
    h = 1.0 / N
    stream = torch.cuda.Stream(device=dev)
    sims = {}
    for s in SCHEMES:
        lam = 0.9 * LAMBDA_MAX[s]
        sims[s] = w.Wave2D(N, N, h, lam * h, scheme=s, bc=BC_PERIODIC, dtype=w.F32, stream=stream.cuda_stream)
    du0 = torch.from_numpy(u0).to(dev)
    dv0 = torch.from_numpy(v0).to(dev)
    torch.cuda.synchronize(dev)
    # Autotune each handle once on its own data (outside the timed region).
    tuned = {}
    for s in SCHEMES:
        sims[s].first_step(du0, dv0)
        if args.fixed_tuning:  # the autotuner's choice on the measured runs
            kname, rows, depth = FIXED_TUNING[s]
            kern = w.KERNEL_STREAM if kname == "stream" else w.KERNEL_TEMPORAL
            sims[s].set_tuning(kernel=kern, temporal_t=depth, tile_h=rows)
            best = w.wave2d_tune(kern, rows, depth, -1, 0)
        else:
            best = sims[s].autotune(steps=64)
        tuned[s] = {"kernel": KSHORT[best.kernel],
                    "temporal_t": best.temporal_t, "tile_h": best.tile_h, "ctas_per_sm": best.ctas_per_sm}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MiB > L2
    torch.cuda.synchronize(dev)
    results = {}

    def one_step(timing=None):
        with torch.cuda.stream(stream):
            flush.zero_()  # evict the previous step's levels from L2
        for s in SCHEMES:
            sims[s].first_step(du0, dv0)
            if timing is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            sims[s].step_n(STEPS_PER_SCHEME - 1)
            if timing is not None:
                e1.record(stream)
                timing.append((s, e0, e1))
            results[s] = sims[s].error_vs_exact()  # FP64 norm -> host (synchronises)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        one_step()
    barrier()
    timing = []
    c0 = w.launch_count()
    with ClockSampler(local_rank) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(args.steps):
            one_step(timing)
        t_end.record(stream)
        barrier()
    launches = w.launch_count() - c0
    elapsed = t_start.elapsed_time(t_end) / 1e3
    stepn_s = sum(a.elapsed_time(b) for _, a, b in timing) / 1e3

    def time_levels(sim, n_levels, reps=1):
        """Event time of n_levels two-steps on the handle's stream."""
        sim.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            sim.step_n(n_levels)
        e1.record(stream)
        sim.sync()
        return e0.elapsed_time(e1) / 1e3

    # Per-launch durations of the kernels inside step_n (after the timed
    # region): the one-step TMA kernel that finishes runs of a multi-level
    # kernel (temporal or streaming), and which kernel each handle uses.
    MULTI = (w.KERNEL_TEMPORAL, w.KERNEL_STREAM)
    kinfo = {}
    one_step = {}
    for s in SCHEMES:
        info = sims[s].info()
        kinfo[s] = (info.kernel, info.temporal_t)
        if info.kernel in MULTI:
            sims[s].set_tuning(kernel=w.KERNEL_TMA, use_graph=0)
            one_step[s] = time_levels(sims[s], 200) / 200
            sims[s].set_tuning(kernel=info.kernel, temporal_t=info.temporal_t, tile_h=tuned[s]["tile_h"])
        else:
            one_step[s] = None

    # End to end through the public API with host buffers (pinned), copies
    # timed: one handle per scheme on its own stream (the same tuning as the
    # timed handles), so that one scheme's host -> device upload overlaps the
    # other's stepping; every step uploads both schemes' inputs and reads both
    # norms back.
    pu0 = torch.from_numpy(u0).pin_memory()
    pv0 = torch.from_numpy(v0).pin_memory()
    e2e_streams = {s: torch.cuda.Stream(device=dev) for s in SCHEMES}
    e2e_sims = {}
    for s in SCHEMES:
        lam = 0.9 * LAMBDA_MAX[s]
        e2e_sims[s] = w.Wave2D(N, N, h, lam * h, scheme=s, bc=BC_PERIODIC, dtype=w.F32,
                               stream=e2e_streams[s].cuda_stream)
        kern = {"stream": w.KERNEL_STREAM, "temporal": w.KERNEL_TEMPORAL, "tma": w.KERNEL_TMA,
                "simple": w.KERNEL_SIMPLE, "persistent": w.KERNEL_PERSISTENT}[tuned[s]["kernel"]]
        e2e_sims[s].set_tuning(kernel=kern, temporal_t=tuned[s]["temporal_t"], tile_h=tuned[s]["tile_h"],
                               ctas_per_sm=tuned[s]["ctas_per_sm"])

    def e2e_step():
        with torch.cuda.stream(stream):
            flush.zero_()
        for s in SCHEMES:
            e2e_streams[s].wait_stream(stream)   # after the L2 flush
        for s in SCHEMES:
            e2e_sims[s].first_step(pu0, pv0)     # host -> device copy inside the call
            e2e_sims[s].step_n(STEPS_PER_SCHEME - 1)
        for s in SCHEMES:
            results[s] = e2e_sims[s].error_vs_exact()  # device -> host norms

    e2e_step()  # warm-up of the new handles (staging pools, first launches)
    barrier()
    e2e_steps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_elapsed = time.perf_counter() - t0

    # Error of the benchmark's FP32 result (the last step's final level, k =
    # 2000) against an FP64 run of the same inputs and levels on the GPU (the
    # FP64 path matches the CPU oracle to 1e-12 in the parity tests).
    result_error = {}
    if not args.no_extras:
        for s in SCHEMES:
            lam = 0.9 * LAMBDA_MAX[s]
            with w.Wave2D(N, N, h, lam * h, scheme=s, bc=BC_PERIODIC, dtype=w.F64,
                          stream=stream.cuda_stream) as ref64:
                ref64.first_step(du0, dv0)
                ref64.step_n(STEPS_PER_SCHEME - 1)
                l2, linf = e2e_sims[s].diff_norms(ref64)  # the end-to-end run's final level, k = 2000
            result_error[str(s)] = {"rel_l2": l2, "rel_linf": linf}
    for s in SCHEMES:
        e2e_sims[s].close()

    elapsed, e2e_elapsed = reduce_max([elapsed, e2e_elapsed], dev)
    pts_step = len(SCHEMES) * STEPS_PER_SCHEME * N * N
    value = whole_job_value(args.steps * pts_step, world, elapsed)
    e2e_value = whole_job_value(e2e_steps * pts_step, world, e2e_elapsed)
    for s in SCHEMES:
        sims[s].close()
    if rank != 0:
        return None

    peak, peak_src = measured_peaks()
    per_scheme_stepn = {s: sum(a.elapsed_time(b) for ss, a, b in timing if ss == s) / 1e3 for s in SCHEMES}
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or 2070.0
    spec_alu = sms * 128 * mhz * 1e6 / 1e12
    # The FP32-pipe peak measured on this GPU (wave2d_alu_peaks: the best of
    # scalar FMA, packed f32x2 FMA and add throughput), the denominator of the
    # temporal kernels' ALU roofline; the spec figure rides along.
    pk = w.alu_peaks(stream.cuda_stream)
    alu_peak = max(pk.fp32_fma, pk.fp32_fma2, pk.fp32_add) / 1e12
    alu_measured = {"fp32_fma_tops": round(pk.fp32_fma / 1e12, 3), "fp32_fma2_tops": round(pk.fp32_fma2 / 1e12, 3),
                    "fp32_add_tops": round(pk.fp32_add / 1e12, 3), "fp64_fma_tops": round(pk.fp64_fma / 1e12, 4),
                    "unit": "T lane operations/s (FMA = 1)", "spec_fp32_tops": round(spec_alu, 2),
                    "spec": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}
    # One roofline per kernel in step_n, over the launches of the schemes that
    # use it.  step_n(1999) of a multi-level kernel = floor(1999 / T) launches
    # of T levels + (1999 mod T) one-step launches (timed separately above).
    groups = {}
    for s in SCHEMES:
        kern, T = kinfo[s]
        if kern not in MULTI:
            T = 1
        groups.setdefault((KNAME[kern], T), []).append(s)
    rooflines = []
    for (kname, T), ss in groups.items():
        total = sum(per_scheme_stepn[s] for s in ss)
        if T > 1:
            total -= sum(args.steps * ((STEPS_PER_SCHEME - 1) % T) * one_step[s] for s in ss)
        n_launch = len(ss) * args.steps * ((STEPS_PER_SCHEME - 1) // T)
        avg_launch = total / n_launch
        alg_bytes = (16 if T > 1 else 12) * N * N  # read the two levels, write two (one for one step)
        achieved = alg_bytes / avg_launch / 1e9
        per = [NCU_TRAFFIC.get((kname, kernel_source_hash(kname), s, tuned[s]["tile_h"] if T > 1 else 0, T))
               for s in ss]
        traffic = int(sum(per) / len(per)) if all(per) else None  # mean over the schemes' launches
        label = f"{kname} (FP32, T={T}, {'/'.join(str(s) for s in ss)}-point)"
        hbm_view = {"bound": "hbm", "kernel": label, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "peak_source": peak_src,
                    "algorithmic_bytes_per_launch": alg_bytes, "levels_per_launch": T,
                    "avg_launch_us": round(avg_launch * 1e6, 3), "traffic": traffic,
                    "unblocked_equivalent_gbs": round(12 * T * N * N / avg_launch / 1e9, 1),
                    "share_of_step_n": round(sum(per_scheme_stepn[s] for s in ss) / stepn_s, 4)}
        if T == 1:
            rooflines.append(hbm_view)
            continue
        # Temporal blocking takes the kernel off HBM (DRAM 31-44 % busy in
        # ncu); its limit is the FP32 pipe.  Algorithmic work: the two-step as
        # written, FP32_OPS per node-update, T levels per launch, the schemes'
        # launches equally many.  Peak: one FP32 add, multiply or fused
        # multiply-add per lane per clock, 128 lanes per SM.
        alg_ops = T * N * N * sum(FP32_OPS[s] for s in ss) / len(ss)
        alu = alg_ops / avg_launch / 1e12
        rooflines.append({"bound": "alu", "kernel": label, "achieved": round(alu, 2), "peak": round(alu_peak, 2),
                          "unit": "TFLOP/s", "frac": round(alu / alu_peak, 4),
                          "flop": "one FP32 add, multiply or fused multiply-add (one FP32-pipe lane slot)",
                          "peak_source": "measured on this GPU (wave2d_alu_peaks: best of scalar FMA, packed "
                                         "f32x2 FMA and add lane-operation rates)",
                          "frac_of_spec": round(alu / spec_alu, 4),
                          "algorithmic_flop_per_launch": int(alg_ops), "levels_per_launch": T,
                          "avg_launch_us": round(avg_launch * 1e6, 3), "traffic": traffic,
                          "share_of_step_n": hbm_view["share_of_step_n"], "hbm": hbm_view})
    rooflines.sort(key=lambda r: -r["share_of_step_n"])
    roofline = dict(rooflines[0])  # the dominant kernel
    if len(rooflines) > 1:
        roofline["other_kernels"] = rooflines[1:]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "G point-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": N, "schemes": list(SCHEMES),
                   "time_levels_per_scheme": STEPS_PER_SCHEME, "boundary": "periodic",
                   "point_updates_per_step": pts_step, "l2_flush_between_steps": True,
                   "autotuned": {str(s): tuned[s] for s in SCHEMES},
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "per_scheme_ms_per_level": {str(s): round(per_scheme_stepn[s] / (args.steps * (STEPS_PER_SCHEME - 1)) * 1e3, 5)
                                    for s in SCHEMES},
        "e2e": {"value": round(e2e_value, 3), "unit": "G point-updates/s",
                "h2d_bytes_per_step": len(SCHEMES) * 2 * 8 * N * N,
                "d2h_bytes_per_step": len(SCHEMES) * (8 * 8 + 4),
                "schedule": "one handle per scheme on its own stream: each scheme's upload and stepping "
                            "overlap the other's (the device-timed value runs the schemes back to back on "
                            "one stream, for the per-kernel roofline)"},
        "gpu_launches": launches,
        "one_step_kernel": ({"kernel": "k2_tma", "avg_launch_us": {str(s): round(one_step[s] * 1e6, 3) for s in SCHEMES},
                             "frac": {str(s): round(12 * N * N / one_step[s] / 1e9 / peak, 4) for s in SCHEMES},
                             "algorithmic_bytes_per_launch": 12 * N * N,
                             "traffic": NCU_TRAFFIC.get(("k2_tma", kernel_source_hash("k2_tma"), 13, 0, 1))}
                            if all(one_step[s] for s in SCHEMES) else None),
        "clocks": clocks,
        "alu_peaks_measured": alu_measured,
        "result_norms": {str(s): [results[s][0], results[s][1]] for s in SCHEMES},
        "result_error_vs_fp64": ({"reference": "FP64 run of the same inputs and levels on the GPU (the FP64 path "
                                               "matches the CPU oracle to 1e-12 in the parity tests)",
                                  **result_error} if result_error else None),
    }
    if world == 1 and not args.no_extras:
        line["fp64_5point_256"] = measure_small_fp64(w, torch)
        line["batched"] = measure_batched(w, torch)
        line["served"] = measure_served(w, torch)
        line["derived_schemes"] = measure_derived(w, torch, u0, v0, peak)
        plain_us = {s: line["per_scheme_ms_per_level"][str(s)] * 1e3 for s in SCHEMES}
        line["fp32_difference_sums"] = measure_diff_sums(w, torch, u0, v0, peak, plain_us)
        if args.precision != "off":
            line["precision"] = measure_precision(w, torch, args.precision)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = time_oracle(u0, v0, args.cpu_budget)
        if not args.no_extras:
            line["oracle_timings"] = time_oracle_table(u0, v0)
    return line


def measure_batched(w, torch):
    """512 uneven instances (sizes log-uniform 64..1024, mixed schemes, Courant
    numbers and 100..2000 steps, zero boundary, centred Gaussian pulse): one
    batched run per repetition vs the plain per-grid launch loop."""
    from initial_data import BC_ZERO, batch_instances, instance_ic
    insts = batch_instances(512, seed=4)
    data = [instance_ic(i) for i in insts]
    du = [torch.from_numpy(d[0]).cuda() for d in data]
    dv = [torch.from_numpy(d[1]).cuda() for d in data]
    steps = [i.steps for i in insts]
    pts = sum(i.n * i.n * (i.steps + 1) for i in insts)
    stream = torch.cuda.Stream()
    sims = [w.Wave2D(i.n, i.n, h, i.lam * h, scheme=i.scheme, bc=BC_ZERO, dtype=w.F32, stream=stream.cuda_stream)
            for i, (_, _, h) in zip(insts, data)]
    b = w.Batch(sims)
    b.first_step(du, dv)
    best = b.autotune(steps, probe_steps=32)
    b.first_step(du, dv)
    b.run(steps)            # builds and captures the run
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        b.first_step(du, dv)
        b.run(steps)
        norms = b.norms()
    torch.cuda.synchronize()
    batched = (time.perf_counter() - t0) / reps
    for sm in sims:
        sm.set_tuning(kernel=w.KERNEL_AUTO, use_graph=0)
    t0 = time.perf_counter()
    for sm, a, c, n in zip(sims, du, dv, steps):
        sm.first_step(a, c)
        sm.step_n(n)
    plain_norms = [sm.error_vs_exact()[0] for sm in sims]
    torch.cuda.synchronize()
    plain = time.perf_counter() - t0
    agree = max(abs(x - y[0]) / y[0] for x, y in zip(plain_norms, norms))
    b.close()
    for sm in sims:
        sm.close()
    return {"workload": "512 instances, n log-uniform 64..1024 (seed 4), schemes 5/9/13, lambda U(0.3, 0.9 max), "
                        "100..2000 steps, FP32, zero boundary, centred Gaussian pulse",
            "node_updates": pts, "value": round(pts / batched / 1e9, 2), "unit": "G point-updates/s",
            "ms": round(batched * 1e3, 2), "plain_loop_value": round(pts / plain / 1e9, 2),
            "plain_loop_ms": round(plain * 1e3, 1), "speedup_vs_plain": round(plain / batched, 2),
            "kernel": KSHORT.get(best.kernel), "quantum": best.temporal_t, "tile_h": best.tile_h,
            "max_rel_norm_diff_vs_plain": agree,
            "timing": "host wall clock around first step + run + norms to host, 3 repetitions"}


def measure_served(w, torch):
    """Poisson stream of 2000 requests at 200 / s (sizes log-uniform
    128..2048, mixed schemes, Courant numbers and 100..5000 steps, FP32, zero
    boundary, Gaussian pulse), 16 GiB budget: latency, throughput and GPU
    busy fraction; the same requests all at once (capacity); and the same
    whole stream as sequential plain launches, each request creating its
    handle and its pulse on the device as the server does (equal work)."""
    import numpy as np
    from initial_data import request_stream
    reqs = request_stream(count=2000, seed=5)

    def serve(paced):
        with w.Server(budget_bytes=16 << 30, max_resident=4096, quantum=64) as srv:
            t0 = time.perf_counter()
            for i, rq in enumerate(reqs):
                if paced:
                    d = t0 + rq.arrival_s - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                n = rq.inst.n
                h = 1.0 / (n + 1)
                srv.submit(n, n, h, rq.inst.lam * h, rq.inst.steps, scheme=rq.inst.scheme,
                           pulse=(1.0, 0.5, 0.5, 0.05), tag=i)
            srv.drain(3600)
            comps = srv.poll(max_n=len(reqs) + 8)
            st = srv.stats()
        lat = np.array([c.t_done - c.t_submit for c in comps])
        wall = max(c.t_done for c in comps) - min(c.t_submit for c in comps)
        assert len(comps) == len(reqs) and all(c.status == 0 for c in comps)
        return lat, wall, st

    pts = sum(r.inst.n ** 2 * (r.inst.steps + 1) for r in reqs)
    lat, wall, st = serve(True)
    _, wall_sat, st_sat = serve(False)
    # sequential plain launches over the whole stream
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for rq in reqs:
            n = rq.inst.n
            h = 1.0 / (n + 1)
            x = (torch.arange(n, dtype=torch.float64, device="cuda") + 1) * h
            g = torch.exp(-(x - 0.5) ** 2 / (2 * 0.05 ** 2))
            u0 = torch.outer(g, g)
            v0 = torch.zeros_like(u0)
            with w.Wave2D(n, n, h, rq.inst.lam * h, scheme=rq.inst.scheme, dtype=w.F32,
                          stream=stream.cuda_stream) as sm:
                sm.set_tuning(use_graph=0)
                sm.first_step(u0, v0)
                sm.step_n(rq.inst.steps)
                sm.error_vs_exact()
    torch.cuda.synchronize()
    seq = pts / (time.perf_counter() - t0) / 1e9
    return {"workload": "2000 Poisson requests at 200/s (seed 5), n log-uniform 128..2048, schemes 5/9/13, "
                        "100..5000 steps, FP32, zero boundary, Gaussian pulse, 16 GiB budget, quantum 64",
            "node_updates": pts, "offered_value": round(pts / reqs[-1].arrival_s / 1e9, 2),
            "value": round(pts / wall / 1e9, 2), "unit": "G point-updates/s",
            "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
            "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
            "gpu_busy_fraction": round(st.gpu_busy_s / wall, 3),
            "max_resident": st.max_resident_seen, "rounds": st.rounds,
            "saturated_value": round(pts / wall_sat / 1e9, 2),
            "saturated_gpu_busy_fraction": round(st_sat.gpu_busy_s / wall_sat, 3),
            "sequential_plain_value": round(seq, 2),
            "saturated_speedup_vs_sequential_plain": round(pts / wall_sat / 1e9 / seq, 2),
            "sequential_plain": "the whole stream, one request after another: handle created, Gaussian pulse "
                                "generated on the device, first step, steps, norms to host, handle destroyed",
            "latency": "submission to norms on the host (library steady clock)"}


PRECISION_SCOPES = {
    "full": "N = 512..8192, schemes 5/9/13, modes (1,0), (3,4), (N/32,N/64); FP64, FP32, FP32 difference form, "
            "FP32x2; FP64 the reference",
    "bounded": "N <= 2048: schemes 5/9/13, modes (1,0), (3,4), (N/32,N/64), FP64/FP32/FP32 difference form/FP32x2, "
               "FP64 the reference; 4096^2: every scheme and mode, FP32/difference form/FP32x2, FP32x2 the "
               "reference; 8192^2: 9- and 13-point, modes (1,0) and (256,128), FP32/difference form/FP32x2, "
               "FP32x2 the reference"}


def precision_cases(scope: str):
    """The plane-wave precision sweep: (N, scheme, (m1, m2), dtypes, reference).

    Every case runs a periodic plane wave cos(k.x - c|k| t), k = 2 pi (m1, m2),
    on the N^2 unit square, lambda = 0.9 of the scheme's limit, 10^4 two-steps
    after the first step.  dtypes are "f64", "f32", "f32_diff_form" (FP32 with
    WAVE2D_DIFF_FORM) and "f32x2"; the reference is the dtype the others are
    compared with (FP64 where it runs; FP32x2, which tracks FP64 to ~1e-11,
    above 2048^2, where an FP64 run of 10^4 levels takes 6-24 s per case).
      full:    N = 512 .. 8192, schemes 5, 9, 13, modes (1,0), (3,4),
               (N/32, N/64), all four dtypes, FP64 the reference.
      bounded: N <= 2048 as full; 4096^2 every scheme and mode without FP64;
               8192^2 the 9- and 13-point schemes, modes (1,0) and (N/32, N/64),
               without FP64."""
    out = []
    for n in (512, 1024, 2048, 4096, 8192):
        modes = [(1, 0), (3, 4), (n // 32, n // 64)]
        schemes = (5, 9, 13)
        if scope == "full" or n <= 2048:
            dts, ref = ("f64", "f32", "f32_diff_form", "f32x2"), "f64"
        else:
            dts, ref = ("f32", "f32_diff_form", "f32x2"), "f32x2"
            if n == 8192:
                schemes, modes = (9, 13), [(1, 0), (n // 32, n // 64)]
        for sc in schemes:
            for m in modes:
                out.append((n, sc, m, dts, ref))
    return out


def measure_precision(w, torch, scope: str, steps: int = 10000):
    """Error of every storage mode over 10^4 steps of a periodic plane wave
    (the precision sweep): relative L2 and L-infinity against the exact PDE
    solution (FP64 norms on the device) and against the reference run of the
    same case (wave2d_diff_norms), and the time per level (CUDA events around
    step_n on the handle's stream)."""
    import math
    from initial_data import BC_PERIODIC, LAMBDA_MAX, plane_wave_ic
    flags = {"f64": (w.F64, 0), "f32": (w.F32, 0), "f32_diff_form": (w.F32, w.DIFF_FORM), "f32x2": (w.F32X2, 0)}
    rows = []
    t_start = time.perf_counter()
    ic_cache = {}
    for n, sc, (m1, m2), dts, ref_dt in precision_cases(scope):
        h = 1.0 / n
        lam = 0.9 * LAMBDA_MAX[sc]
        tau = lam * h
        k1, k2 = 2 * math.pi * m1, 2 * math.pi * m2
        key = (n, m1, m2)
        if key not in ic_cache:
            ic_cache.clear()
            u0, v0 = plane_wave_ic(n, n, h, k1, k2, BC_PERIODIC)
            ic_cache[key] = (torch.from_numpy(u0).cuda(), torch.from_numpy(v0).cuda())
            del u0, v0
        du0, dv0 = ic_cache[key]
        ex = w.exact(w.EXACT_PLANE, amp=1.0, k1=k1, k2=k2, x_off=0.0)
        stream = torch.cuda.Stream()
        sims = {}
        try:
            for dt in [ref_dt] + [d for d in dts if d != ref_dt]:
                dtype, fl = flags[dt]
                sim = w.Wave2D(n, n, h, tau, scheme=sc, bc=BC_PERIODIC, dtype=dtype, flags=fl,
                               stream=stream.cuda_stream)
                sims[dt] = sim
                sim.first_step(du0, dv0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step_n(steps)
                e1.record(stream)
                l2, linf, _ = sim.error_vs_exact(ex)
                row = {"N": n, "scheme": sc, "mode": [m1, m2], "dtype": dt,
                       "us_per_level": round(e0.elapsed_time(e1) * 1e3 / steps, 3),
                       "kernel": KSHORT.get(sim.info().kernel), "err_exact_l2": l2, "err_exact_linf": linf}
                if dt != ref_dt:
                    rl2, rlinf = sim.diff_norms(sims[ref_dt])
                    row.update({"err_ref_l2": rl2, "err_ref_linf": rlinf, "ref": ref_dt})
                    sim.close()
                    del sims[dt]
                rows.append(row)
        finally:
            for sim in sims.values():
                sim.close()
    ic_cache.clear()
    summary = {}
    for r in rows:
        if "err_ref_l2" not in r:
            continue
        k = f"{r['N']}_{r['dtype']}"
        cur = summary.setdefault(k, {"max_err_ref_l2": 0.0, "max_err_ref_linf": 0.0, "ref": r["ref"]})
        cur["max_err_ref_l2"] = max(cur["max_err_ref_l2"], r["err_ref_l2"])
        cur["max_err_ref_linf"] = max(cur["max_err_ref_linf"], r["err_ref_linf"])
    return {"workload": "periodic plane waves cos(k.x - c|k|t), k = 2 pi (m1, m2), N^2 unit square, "
                        "lambda = 0.9 lambda_max, 10^4 two-steps after the first step",
            "scope": scope, "cases": PRECISION_SCOPES[scope],
            "steps": steps, "seconds": round(time.perf_counter() - t_start, 1),
            "max_error_vs_reference": summary, "rows": rows}


def measure_small_fp64(w, torch):
    """5-point scheme, FP64, 256^2, h = 1/256, c = 1, lambda = 0.5, 200 time
    levels, centred Gaussian pulse (sigma 0.05), v0 = 0, zero boundary: wall
    time of one whole run (first step, 199 two-steps in a CUDA graph, FP64
    norm to the host)."""
    import numpy as np
    from initial_data import BC_ZERO, gaussian_pulse
    n, h, lam = 256, 1.0 / 256, 0.5
    u0 = gaussian_pulse(n, n, h, BC_ZERO, sigma=0.05)
    du = torch.from_numpy(u0).cuda()
    dv = torch.zeros_like(du)
    stream = torch.cuda.Stream()
    with w.Wave2D(n, n, h, lam * h, scheme=5, bc=BC_ZERO, dtype=w.F64, stream=stream.cuda_stream) as sim:
        sim.first_step(du, dv)
        best = sim.autotune(steps=64)
        for _ in range(3):
            sim.first_step(du, dv)
            sim.step_n(199)
            sim.error_vs_exact()
        torch.cuda.synchronize()
        reps = 50
        t0 = time.perf_counter()
        for _ in range(reps):
            sim.first_step(du, dv)
            sim.step_n(199)
            l2, linf, _ = sim.error_vs_exact()
        dt = (time.perf_counter() - t0) / reps
    return {"workload": "5-point, FP64, 256^2, h = 1/256, lambda = 0.5, 200 levels, centred Gaussian, zero boundary",
            "us_per_run": round(dt * 1e6, 1), "value": round(n * n * 200 / dt / 1e9, 3), "unit": "G point-updates/s",
            "kernel": KSHORT.get(best.kernel), "field_l2": l2,
            "timing": "host wall clock per run incl. norm to host, 50 runs"}


def measure_derived(w, torch, u0, v0, peak):
    """Derived schemes (monomial segments m = 24, 28, 45: 21, 25 and 41
    points) on the benchmark grid and inputs, FP32, lambda = 0.9 of each
    scheme's limit: autotuned two-step kernel, 200 levels timed with CUDA
    events on the handle's stream after 20 warm-up levels; HBM roofline at
    12 B per node-update."""
    from initial_data import BC_PERIODIC
    out = {}
    h = 1.0 / N
    for m in (24, 28, 45):
        s = w.derive_scheme(m)
        lam = 0.9 * w.scheme_lambda_max(s)
        stream = torch.cuda.Stream()
        with w.Wave2D(N, N, h, lam * h, scheme=s, bc=BC_PERIODIC, dtype=w.F32, stream=stream.cuda_stream) as sim:
            sim.first_step(u0, v0)
            best = sim.autotune(steps=16)
            sim.step_n(20)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            levels = 200
            e0.record(stream)
            sim.step_n(levels)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3 / levels
        out[str(s.n_points)] = {"segment": m, "lambda": round(lam, 6), "us_per_level": round(sec * 1e6, 2),
                                "value": round(N * N / sec / 1e9, 1), "unit": "G point-updates/s",
                                "kernel": KSHORT.get(best.kernel),
                                "hbm_frac": round(12 * N * N / sec / 1e9 / peak, 3)}
    return out


def measure_diff_sums(w, torch, u0, v0, peak, plain_us=None):
    """The 9- and 13-point schemes in FP32 with WAVE2D_DIFF_SUMS (stencil sums
    from differences to the centre) and with WAVE2D_DIFF_FORM (levels kept as
    u^k and d^k = u^k - u^{k-1}) on the benchmark grid and inputs: autotuned
    two-step kernel, 200 levels timed with CUDA events after 20 warm-up
    levels.  Algorithmic bytes per node-update: 12 (sums) or 16 (form) for a
    one-level kernel, 16 / T for the streaming kernel (two planes read, two
    written per launch of T levels), which is bound by the FP32 pipe, not
    HBM: ``vs_plain`` is the time per level over the plain two-step's on the
    same grid (``plain_us``, from the main measurement)."""
    from initial_data import BC_PERIODIC, LAMBDA_MAX
    out = {}
    h = 1.0 / N
    cases = [(name, flags, bpn, scheme) for (name, flags, bpn) in (("sums", w.DIFF_SUMS, 12), ("form", w.DIFF_FORM, 16))
             for scheme in SCHEMES]
    for name, flags, bpn, scheme in cases:
        lam = 0.9 * LAMBDA_MAX[scheme]
        stream = torch.cuda.Stream()
        with w.Wave2D(N, N, h, lam * h, scheme=scheme, bc=BC_PERIODIC, dtype=w.F32, flags=flags,
                      stream=stream.cuda_stream) as sim:
            sim.first_step(u0, v0)
            best = sim.autotune(steps=16)
            sim.step_n(20)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            levels = 200
            e0.record(stream)
            sim.step_n(levels)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3 / levels
            info = sim.info()
        T = info.temporal_t if info.kernel == w.KERNEL_STREAM else 1
        bytes_per = bpn if T == 1 else 16 / T
        row = {"us_per_level": round(sec * 1e6, 2), "value": round(N * N / sec / 1e9, 1),
               "unit": "G point-updates/s", "kernel": KSHORT.get(info.kernel), "levels_per_launch": T,
               "strip_rows": best.tile_h if T > 1 else None,
               "bytes_per_node_update": round(bytes_per, 3),
               "hbm_frac": round(bytes_per * N * N / sec / 1e9 / peak, 3)}
        if plain_us and plain_us.get(scheme):
            row["vs_plain"] = round(sec * 1e6 / plain_us[scheme], 3)
        out[f"{name}_{scheme}"] = row
    return out


def measure_slabs(n: int = 8192, scheme: int = 13, levels: int = 400, T: int = 4):
    """Row-slab decomposition of one grid (paper_1904_04048_gb300/slab.py),
    all slabs on this GPU: an n^2 periodic grid, FP32, the streaming kernel
    (T levels per launch, 64-row strips), split into P = 1 (the undivided
    handle), 2, 4 and 8 slabs that exchange their R T halo rows (both
    planes, device buffers) after every T levels.  Host wall clock over
    ``levels`` levels after the first step and a warm-up of 2 T levels; the
    slabs advance one after another on the default stream (row copies
    stream-ordered, no host wait per exchange), so the figure is the
    decomposition's cost on one device (halo recomputation, row copies, the
    host's launch work per slab), not a multi-GPU speed."""
    import torch
    from initial_data import BC_PERIODIC, LAMBDA_MAX, pulses_and_noise
    from paper_1904_04048_gb300 import slab
    from paper_1904_04048_gb300 import wave2d as w
    u0, v0 = pulses_and_noise(n, seed=SEED)
    h = 1.0 / n
    lam = 0.9 * LAMBDA_MAX[scheme]
    R = 2 if scheme == 13 else 1
    tune = dict(kernel=w.KERNEL_STREAM, temporal_t=T, tile_h=64, use_graph=0)
    out = {}
    for P in (1, 2, 4, 8):
        sims, runs = [], []
        try:
            for r in range(P):
                plan = slab.plan_slabs(n, n, P, r, R, T, True)
                sim = w.Wave2D(n, plan.ny_local, h, lam * h, scheme=scheme, bc=BC_PERIODIC, dtype=w.F32)
                sim.set_tuning(**tune)
                sims.append(sim)
                runs.append(slab.SlabRun(plan, slab.HandleSolver(sim), device=torch.device("cuda")))
            exch = slab.LocalExchange(sync=False)  # every handle and buffer on the default stream
            slab.first_step(runs, exch, [slab.extended_rows(r.plan, u0) for r in runs],
                            [slab.extended_rows(r.plan, v0) for r in runs])
            slab.step_n(runs, exch, 2 * T)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            slab.step_n(runs, exch, levels)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
        finally:
            for sim in sims:
                sim.close()
        out[str(P)] = {"ms": round(sec * 1e3, 2), "value": round(n * n * levels / sec / 1e9, 1),
                       "unit": "G point-updates/s", "halo_rows_per_slab": 2 * R * T if P > 1 else 0}
    base = out["1"]["value"]
    for v in out.values():
        v["vs_undivided"] = round(v["value"] / base, 3)
    return {"workload": f"{n}^2 periodic, {scheme}-point, FP32, streaming T = {T}, 64-row strips, {levels} "
                        f"levels, slabs exchanging halo rows every T levels, all on one GPU",
            "slabs": out}


def profile_case(kernel: str, scheme: int, segment: int = 28, tile_h: int = 32, depth: int = 4,
                 mode: str = "plain"):
    """A short run of one kernel at the benchmark size, for profiler captures:
    the first step, then a few launches of the named kernel on the
    benchmark's inputs (no timing, no JSON line).  4096^2 FP32 holds about
    0.5 GB on the device.
      k2_tma:      4 one-step launches (the first step comes before them)
      k3_temporal: 3 launches of T = 4 levels, tile_h-row tiles
      k5_stream:   3 launches of T = depth levels, tile_h-row strips
      kc2_tma:     4 one-step launches of a derived scheme (``segment``)
      k2_df2:      4 one-step launches in double-float (FP32x2) storage, the
                   packed two-node kernel (about 0.5 GB on the device)"""
    from initial_data import BC_PERIODIC, LAMBDA_MAX, pulses_and_noise
    from paper_1904_04048_gb300 import wave2d as w
    u0, v0 = pulses_and_noise(N, seed=SEED)
    h = 1.0 / N
    if kernel == "kc2_tma":
        scheme = w.derive_scheme(segment)
        lam = 0.9 * w.scheme_lambda_max(scheme)
    else:
        lam = 0.9 * LAMBDA_MAX[scheme]
    flags = {"plain": 0, "sums": w.DIFF_SUMS, "form": w.DIFF_FORM}[mode]
    dtype = w.F32X2 if kernel == "k2_df2" else w.F32
    with w.Wave2D(N, N, h, lam * h, scheme=scheme, bc=BC_PERIODIC, dtype=dtype, flags=flags) as sim:
        if kernel == "k2_df2":
            sim.set_tuning(kernel=w.KERNEL_SIMPLE, use_graph=0)
            levels = 4
        elif kernel in ("k2_tma", "kc2_tma"):
            sim.set_tuning(kernel=w.KERNEL_TMA, use_graph=0)
            levels = 4
        elif kernel == "k5_stream":
            sim.set_tuning(kernel=w.KERNEL_STREAM, temporal_t=depth, tile_h=tile_h, use_graph=0)
            levels = 3 * depth
        else:
            sim.set_tuning(kernel=w.KERNEL_TEMPORAL, temporal_t=4, tile_h=tile_h, use_graph=0)
            levels = 12
        sim.first_step(u0, v0)
        sim.step_n(levels)
        sim.sync()
        print(f"profile case {kernel} ({mode}), {sim.info().n_points} points, {N}^2: {levels} levels after the "
              f"first step")


def run_reference(args, rank):
    """The FP64 CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return None
    import oracle
    from initial_data import LAMBDA_MAX, pulses_and_noise
    u0, v0 = pulses_and_noise(N, seed=SEED)
    threads = oracle.set_threads(os.cpu_count() or 1)
    h = 1.0 / N
    levels = args.ref_levels
    def one():
        for s in SCHEMES:
            lam = 0.9 * LAMBDA_MAX[s]
            oracle.run(s, u0, v0, lam, lam * h, levels, bc=oracle.BC_PERIODIC)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    pts = args.steps * len(SCHEMES) * levels * N * N
    v = pts / dt / 1e9
    sample = (f"each step: both schemes on the full {N}^2 grid for {levels} time levels "
              f"(the full workload has {STEPS_PER_SCHEME})")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "G point-updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": N, "schemes": list(SCHEMES),
                       "time_levels_per_scheme": levels, "boundary": "periodic"},
            "cpu_baseline": {"value": round(v, 5), "unit": "G point-updates/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 5), "unit": "G point-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and served workloads")
    ap.add_argument("--fixed-tuning", action="store_true",
                    help="skip the autotuner (the kernels and rows of FIXED_TUNING, T = 4), e.g. under a profiler")
    ap.add_argument("--ref-levels", type=int, default=4, help="time levels per scheme per reference step")
    ap.add_argument("--precision", choices=["off", "bounded", "full"], default="bounded",
                    help="plane-wave precision sweep over storage modes (see precision_cases)")
    ap.add_argument("--profile-case", choices=["k2_tma", "k3_temporal", "k5_stream", "kc2_tma", "k2_df2"],
                    help="run a short case of one kernel for a profiler capture and exit")
    ap.add_argument("--profile-scheme", type=int, choices=[5, 9, 13], default=13)
    ap.add_argument("--profile-segment", type=int, default=28, help="derived scheme for kc2_tma")
    ap.add_argument("--profile-tile", type=int, default=32, help="rows per tile or strip (k3_temporal, k5_stream)")
    ap.add_argument("--profile-depth", type=int, default=4, help="levels per launch of k5_stream")
    ap.add_argument("--profile-mode", choices=["plain", "sums", "form"], default="plain",
                    help="storage and arithmetic: plain sums, WAVE2D_DIFF_SUMS or WAVE2D_DIFF_FORM")
    ap.add_argument("--slab-probe", action="store_true",
                    help="measure the row-slab decomposition of one 8192^2 grid on this GPU (one JSON line)")
    args = ap.parse_args()
    if args.slab_probe:
        print(json.dumps(measure_slabs()))
        return
    if args.profile_case:
        profile_case(args.profile_case, args.profile_scheme, args.profile_segment, args.profile_tile,
                     args.profile_depth, args.profile_mode)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        args.gpus = world
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            torch.distributed.init_process_group("nccl")
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
