"""Benchmark: lensed images/s on the substructure workload (200x200 grid, supersampling 3,
10,000 truncated-NFW subhalos, EPL + shear, elliptical Sersic, 21x21 Moffat PSF).

One step = one lensed image through the C ABI: lens_sim_image (subhalo constants + the
fused trace/subhalo-sum/Sersic/bin-down kernel) into a device buffer, then
lens_sim_convolve (PSF).  Inputs are device-resident when timing starts; L2 is flushed
(256 MiB write) between steps and only the steps are timed, with CUDA events on the
launching stream.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the baseline arm) on the host cores, each step a
bounded band of image rows, extrapolated to images/s.
Under torchrun (N > 1) every rank simulates its own images (weak scaling, no collective on
the data path); the timed region is the max over ranks.
"""
from __future__ import annotations

import argparse
import gc
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lensed images/s (200², 10k subhalos) vs FP64 oracle; served p50/p99 ms"
UNIT = "images/s"
WORKLOAD = ("substructure image: 200x200 grid at 0.04\", supersampling 3 (360,000 traced points), "
            "EPL + shear, 10,000 truncated-NFW subhalos, elliptical Sersic, 21x21 Moffat PSF, FP32")
N_SYSTEMS = 8            # distinct seeded systems cycled through the steps
# Algorithmic work of one point-subhalo pair, by the form the pair takes.  Far pairs (a unit's
# bounding box beyond 7 max(tau, 1) Rs of the subhalo): dx, dy (2 FADD); r^2 = dx^2 + dy^2 (FMUL,
# FFMA); u = rsqrt(r^2) (1 MUFU); u^2 (FMUL); Horner over the series coefficients; g = p u^2
# (FMUL); alpha += g (dx, dy) (2 FFMA).  With c_0, c_2 .. c_K that is K - 1 Horner FFMA, so
# 8 FFMA + 3 FMUL + 2 FADD = 21 flops (FMA = 2) for the 6-term series (from 7 max(tau, 1) Rs),
# 17 for the 4-term series (from 20), 15 for the 3-term series (from 40).  Marked (near) pairs
# evaluate the 6-term series and the 12-term annulus polynomial (t = a u + b, 11 Horner FFMA,
# one FMUL) for every sample: 21 + 25 = 46 flops (the closed forms of the few samples within
# 4 Rs are not counted).  One MUFU per pair in every form.
FLOPS_BY_FORM = {"near": 46, "series6": 21, "series4": 17, "series3": 15}
FLOPS_PER_PAIR = 21  # the 6-term series formula: the previous single-form ledger, reported beside
KERNEL_SOURCES = ("paper_2606_01547_gb300/csrc/trace.cu", "paper_2606_01547_gb300/csrc/trace_unit.cuh",
                  "paper_2606_01547_gb300/csrc/trace_far.cu", "paper_2606_01547_gb300/csrc/lens_device.cuh",
                  "paper_2606_01547_gb300/csrc/kernels.h")
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "trace_kernel_substructure_200x200_traffic.txt")


INTERP_FLOPS_PER_SAMPLE = 364  # far-field interpolation: 2 x 38 (Lagrange factors) + 288 (tensor sum)


def pair_census(system, kappa: float = 0.0) -> dict:
    """Pairs of a system by the form the trace kernel gives them: the class of each (work unit,
    subhalo) follows from the distance of the unit's sample bounding box to the subhalo, against
    7, 20 and 40 max(tau, 1) Rs (computed here in FP64; the kernel compares FP32 copies, so a
    pair on a boundary may fall on the other side).  With the far-field interpolation (kappa >
    0) an unmarked subhalo at box distance >= kappa x the box's larger half-width is evaluated at
    the 64 nodes instead of the unit's points, and every point adds the interpolation's flops."""
    g = system.grid
    s = g.s
    bw, bh = {1: (24, 12), 2: (12, 6), 3: (8, 4), 4: (6, 3), 5: (5, 2), 6: (4, 2), 7: (5, 1)}.get(s, (2, 2))
    cx, cy, rs, _, rt = system.subhalos.astype(np.float64)
    tm = np.maximum(rt / rs, 1.0) * rs
    counts = {k: 0 for k in FLOPS_BY_FORM}
    extra = {"interp_pairs": 0, "interp_points": 0}

    def coord(c0, j, n, b):
        return c0 + (j - 0.5 * (n - 1) + (b + 0.5) / s - 0.5) * g.dpix

    for by in range((g.ny + bh - 1) // bh):
        for bx in range((g.nx + bw - 1) // bw):
            j1 = min(bx * bw + bw, g.nx) - 1
            i1 = min(by * bh + bh, g.ny) - 1
            npts = (j1 - bx * bw + 1) * (i1 - by * bh + 1) * s * s
            xmin, xmax = coord(g.x0, bx * bw, g.nx, 0), coord(g.x0, j1, g.nx, s - 1)
            ymin, ymax = coord(g.y0, by * bh, g.ny, 0), coord(g.y0, i1, g.ny, s - 1)
            ddx = np.maximum(np.maximum(xmin - cx, cx - xmax), 0.0)
            ddy = np.maximum(np.maximum(ymin - cy, cy - ymax), 0.0)
            dist = np.hypot(ddx, ddy)
            rho = dist / tm
            interp = (rho >= 7) & (dist >= kappa * 0.5 * max(xmax - xmin, ymax - ymin)) if kappa > 0 else \
                np.zeros_like(rho, bool)
            w = np.where(interp, 64, npts)
            counts["near"] += int((w * (rho < 7)).sum())
            counts["series6"] += int((w * ((rho >= 7) & (rho < 20))).sum())
            counts["series4"] += int((w * ((rho >= 20) & (rho < 40))).sum())
            counts["series3"] += int((w * (rho >= 40)).sum())
            if kappa > 0:
                extra["interp_pairs"] += npts * int(interp.sum())
                extra["interp_points"] += npts
    total = sum(counts.values())
    flops = sum(counts[k] * FLOPS_BY_FORM[k] for k in counts) + extra["interp_points"] * INTERP_FLOPS_PER_SAMPLE
    out = {"pairs": total, "fractions": {k: v / total for k, v in counts.items()},
           "flops": flops, "flops_per_pair": flops / total}
    if kappa > 0:
        out["interpolated_pairs"] = extra["interp_pairs"]
    return out


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments, trailing blanks and empty lines."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_hash() -> str:
    """Hash of the trace kernel's sources as code (comments and blank lines left out), so that a
    profile capture stays matched to the kernel across comment edits but not code changes."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, p)).read()).encode())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------- multi-rank helpers
def rank_seeds(rank: int, n: int = N_SYSTEMS):
    """Seeds of the systems one rank simulates: disjoint across ranks (replicas, weak scaling)."""
    return [1000 + rank * n + i for i in range(n)]


def max_over_ranks(value: float, device, world: int) -> float:
    """The timed region of a multi-rank run is the slowest rank's."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- clocks
REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 3:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[2], 16) if parts[2].startswith("0x") else int(parts[2])
            except ValueError:
                continue
            for b, name in REASON_BITS.items():
                if bits & b:
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arm
def oracle_sample(system, budget_s: float, max_rows: int):
    """Time the FP64 oracle on bands of rows of one image until budget_s or max_rows."""
    import oracle
    oracle.build()
    nx, ny = system.grid.nx, system.grid.ny
    rows, t_total = 0, 0.0
    band = 2
    r = ny // 3
    while rows < max_rows and t_total < budget_s:
        b = min(band, max_rows - rows)
        r0 = (r + rows) % (ny - b)
        t0 = time.perf_counter()
        oracle.image_rows(system, r0, r0 + b)
        t_total += time.perf_counter() - t0
        rows += b
        band = min(band * 2, 32)
    # the PSF step on the full image is timed once and pro-rated
    img = np.random.default_rng(0).random((ny, nx))
    t0 = time.perf_counter()
    oracle.convolve(img, system.psf)
    t_conv = time.perf_counter() - t0
    t_image = t_total * ny / rows + t_conv
    return 1.0 / t_image, rows, oracle.nthreads()


def run_reference(args, rank: int) -> None:
    if rank != 0:
        return
    from paper_2606_01547_gb300 import workloads as W
    system = W.substructure_system(1000)
    # the whole run (warm-up + timed steps) is held to about --ref-budget-s of oracle work
    per_step = max(0.05, args.ref_budget_s / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(system, per_step, 2)
    vals, rows_tot, cores = [], 0, 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, rows, cores = oracle_sample(system, per_step, 200)
        vals.append(v)
        rows_tot += rows
    elapsed = time.perf_counter() - t0
    value = statistics.median(vals)
    sample = (f"{rows_tot} unconvolved rows of 200 over {args.steps} steps (bands of rows of one "
              f"200x200 s=3 image, 10k subhalos) + one full 21x21 convolution per step; extrapolated")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "arm": "FP64 C++ oracle on host cores"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank: int, world: int, local_rank: int) -> None:
    import torch
    import torch.distributed as dist

    from paper_2606_01547_gb300 import lenssim
    from paper_2606_01547_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sim = lenssim.Simulator(device=local_rank)
    systems = [W.substructure_system(seed) for seed in rank_seeds(rank)]
    keep = []
    cs = []
    for s in systems:
        sub_d = torch.from_numpy(s.subhalos).to(dev)
        keep.append(sub_d)
        c = sim.system_struct(s, keep, subhalos=sub_d, use_psf=False)
        cs.append(c)
    psf_id = sim.register_psf(systems[0].psf)
    nx = ny = systems[0].grid.nx
    raw = torch.empty((ny, nx), device=dev)
    out = torch.empty((ny, nx), device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2
    stream = torch.cuda.current_stream()
    sptr = int(stream.cuda_stream)
    L = lenssim.lib()
    import ctypes
    raw_ptrs = (ctypes.c_void_p * 1)(raw.data_ptr())

    def step(i):
        c = cs[i % N_SYSTEMS]
        rc = L.lens_sim_image(sim.h, ctypes.byref(c), 1, raw_ptrs, sptr)
        if rc:
            raise lenssim.LensSimError(rc, sim.last_error())
        return c

    def conv():
        rc = L.lens_sim_convolve(sim.h, raw.data_ptr(), 1, ny, nx, psf_id, out.data_ptr(), sptr)
        if rc:
            raise lenssim.LensSimError(rc, sim.last_error())

    if args.far_field > 0:
        sim.set_far_field(args.far_field)
    if args.variant >= 0:  # fixed variant (profiling runs)
        sim.set_variant(args.variant)
        tune = {"variant": args.variant, "name": lenssim.TRACE_VARIANTS[args.variant], "ms": None}
    else:
        tune = sim.autotune(systems[0], reps=3, use_cache=False)  # untimed: picks the trace launch variant
    for i in range(args.warmup):
        flush.fill_(float(i))
        step(i)
        conv()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i + 1))
            e0, e1, e2 = ev[i]
            e0.record(stream)
            step(i)
            e1.record(stream)
            conv()
            e2.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    step_ms = [e0.elapsed_time(e2) for e0, e1, e2 in ev]
    trace_ms = [e0.elapsed_time(e1) for e0, e1, e2 in ev]
    # The timed region (K steps of ~2 ms) is shorter than the 200 ms sampling period, so the
    # clocks are also sampled over an untimed repeat of the same step lasting --clock-soak-s.
    soak_steps = 0
    with ClockSampler(local_rank) as clk_soak:
        t_end = time.perf_counter() + args.clock_soak_s
        while time.perf_counter() < t_end:
            for _ in range(25):
                step(soak_steps)
                conv()
                soak_steps += 1
            torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(step_ms), dev, world)
    value = throughput(args.steps, world, total_ms / 1000.0)

    # dominant kernel: subhalo constants + fused trace kernel (the launch before the PSF)
    pairs = systems[0].pairs()
    avg_trace_s = statistics.mean(trace_ms) / 1000.0
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    clocks = clk.summary()
    clocks["soak"] = dict(clk_soak.summary(), steps=soak_steps, seconds=args.clock_soak_s)
    max_mhz = clocks["sm_max_mhz"] or 2070.0
    peak_tflops = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    # measured pipe rates per SM and SM clock (after the timed region): the derived FP32 peak's
    # 128 lanes checked, and the MUFU rate the reciprocal square root of every pair draws on
    rates = sim.pipe_rates()
    census = pair_census(systems[0], args.far_field)
    achieved = census["flops"] / avg_trace_s / 1e12
    traffic = None
    if os.path.exists(PROFILE_TRAFFIC):
        prof = dict(l.split(": ", 1) for l in open(PROFILE_TRAFFIC).read().splitlines()
                    if ": " in l and not l.startswith("#"))
        if (prof.get("kernel_hash") == kernel_hash() and prof.get("variant") == tune["name"]
                and args.far_field <= 0):
            traffic = int(prof["traffic_bytes_per_launch"])
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "kernel": f"fused trace kernel, launch variant {tune['name']} (+ tnfw_prep)",
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz (derived, FP32 FMA)",
                "frac_at_median_clock": (achieved / (sms * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
                                         if clocks["sm_mhz"] else None),
                "pairs_per_s": pairs / avg_trace_s, "flops_per_pair": census["flops_per_pair"],
                "pair_forms": census["fractions"], "flops_by_form": FLOPS_BY_FORM,
                "frac_21_flop_ledger": (pairs * FLOPS_PER_PAIR / avg_trace_s / 1e12 / peak_tflops
                                        if args.far_field <= 0 else None),
                "trace_ms": avg_trace_s * 1e3,
                "pipe_rates_per_sm_clock": rates,
                "frac_of_measured_fp32": achieved / (sms * rates["fp32_lane_ops_ffma2"] * 2 * max_mhz * 1e6 / 1e12),
                # SFU: one MUFU.RSQ per evaluated pair against the measured rsqrt rate
                "sfu": {"mufu_per_s": census["pairs"] / avg_trace_s,
                        "peak_per_s": sms * rates["mufu_rsqrt"] * max_mhz * 1e6,
                        "peak_basis": f"{sms} SMs x {rates['mufu_rsqrt']:.2f} rsqrt.approx results per clock "
                                      f"(measured, lens_sim_pipe_rates) x {max_mhz:.0f} MHz",
                        "frac": census["pairs"] / avg_trace_s / (sms * rates["mufu_rsqrt"] * max_mhz * 1e6)}}
    if args.far_field > 0:
        roofline["evaluated_pairs"] = census["pairs"]
        roofline["interpolated_pair_fraction"] = census["interpolated_pairs"] / pairs
        roofline["pairs_per_s_note"] = "pairs of the exact sum per second (the work the interpolation stands in for)"

    # e2e: the public call with HOST buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        sub_h = [torch.from_numpy(s.subhalos).pin_memory() for s in systems]
        out_h = torch.empty((ny, nx), dtype=torch.float32).pin_memory()
        keep2 = []
        cs_h = []
        for s, sh in zip(systems, sub_h):
            c = sim.system_struct(s, keep2, subhalos=sh, use_psf=True)
            cs_h.append(c)
        out_ptrs = (ctypes.c_void_p * 1)(out_h.data_ptr())

        def e2e_step(i):
            rc = L.lens_sim_image(sim.h, ctypes.byref(cs_h[i % N_SYSTEMS]), 1, out_ptrs, sptr)
            if rc:
                raise lenssim.LensSimError(rc, sim.last_error())

        for i in range(args.warmup):
            e2e_step(i)
        torch.cuda.synchronize()
        tsum = 0.0
        for i in range(args.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step(i)  # H2D subhalos, kernels, D2H image, stream sync
            tsum += time.perf_counter() - t0
        tsum = max_over_ranks(tsum, dev, world)
        e2e = {"value": throughput(args.steps, world, tsum), "unit": UNIT,
               "h2d_bytes_per_step": int(systems[0].subhalos.nbytes),
               "d2h_bytes_per_step": int(ny * nx * 4)}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["psf_conv"] = conv_extra(sim, W, dev)
        extras["psf_fft"] = fft_conv_extra(sim, W, dev)
        extras["subhalo_scaling"] = subhalo_scaling_extra(sim, W, dev)
        extras["batched"] = batched_extra(sim, lenssim, W, dev, args.batch_systems,
                                          single_pairs_per_s=roofline["pairs_per_s"])
        extras["batched_small_systems"] = batched_extra(sim, lenssim, W, dev, args.batch_systems, small=True)
        extras["differentiation"] = grad_extra(sim, W, dev)
        extras["fitting"] = fitting_extra(sim, W, dev)
        extras["serving"] = serving_extra(lenssim, W, args.serve_rates, args.serve_seconds)
        extras["per_config"] = per_config_extra(sim, lenssim, W, dev, args.cpu_budget_s)
        extras["far_field"] = far_field_extra(sim, lenssim, W, dev)  # last: it re-tunes the variant

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, rows, cores = oracle_sample(systems[0], args.cpu_budget_s, 200)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{rows} unconvolved rows of one 200x200 s=3 image (10k subhalos) + one full "
                         f"21x21 convolution, extrapolated to whole images"}
        # the same oracle on one core (a short sample: a few rows)
        import oracle
        oracle.set_threads(1)
        v1, rows1, _ = oracle_sample(systems[0], max(2.0, args.cpu_budget_s / 4), 200)
        oracle.set_threads(cores)
        cpu["one_core"] = {"value": v1, "rows": rows1}

    if rank == 0:
        res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD, "grid": 200, "supersample": 3, "n_subhalos": 10000,
                          "psf": 21, "systems_cycled": N_SYSTEMS,
                          "subhalo_sum": ("exact" if args.far_field <= 0 else
                                          f"far-field interpolation, kappa = {args.far_field:g} (approximate: "
                                          "per-subhalo bound in include/lens_sim.h)"),
                          "l2": "flushed between steps (256 MiB write), steps timed individually",
                          "parallelism": f"replicas x{world}"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
               "autotune": tune, **extras,
               "gpu_launches": 3 * args.steps,
               "gpu": props.name}
        print(json.dumps(res), flush=True)
    sim.close()


def batched_extra(sim, lenssim, W, dev, n_sys: int, small: bool = False, single_pairs_per_s: float = 0.0):
    """Uneven batch (grids 64..256, s 1..3, 0..20,000 subhalos, PSF 5..31): one lens_sim_image
    call (persistent fused launches replayed from a CUDA graph) against a host loop of
    single-system calls with a stream synchronisation per call, on the same device inputs.  The
    batched launch's schedule (persistent kernel form, unit-queue order) is autotuned on the
    batch first.  The pair-rate ceiling is the images/s the batch would reach if all its pairs
    ran at the single-image kernel's pair rate on the benchmark image."""
    import ctypes
    import torch
    if small:  # launch-bound mix: small grids and few subhalos
        systems = W.batched_systems(2025, count=n_sys, max_sub=100, grids=(64,))
    else:
        systems = W.batched_systems(2024, count=n_sys)
    subs = [torch.from_numpy(s.subhalos).to(dev) for s in systems]
    outs = [torch.empty((s.grid.ny, s.grid.nx), device=dev) for s in systems]
    keep = []
    arr = (lenssim.LensSystemC * n_sys)()
    for i, s in enumerate(systems):
        arr[i] = sim.system_struct(s, keep, subhalos=subs[i])
    ptrs = (ctypes.c_void_p * n_sys)(*[o.data_ptr() for o in outs])
    L = lenssim.lib()
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)
    pairs = sum(s.pairs() for s in systems)
    bf, bo = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_float * (2 * len(lenssim.BATCH_FORMS)))()
    rc = L.lens_sim_autotune_batch(sim.h, arr, n_sys, ptrs, 1, ctypes.byref(bf), ctypes.byref(bo), ms, sp)
    if rc:
        raise lenssim.LensSimError(rc, sim.last_error())
    schedule = {"chosen": f"{lenssim.BATCH_FORMS[bf.value]}/{lenssim.BATCH_ORDERS[bo.value]}",
                "ms": {f"{lenssim.BATCH_FORMS[f]}/{lenssim.BATCH_ORDERS[o]}": float(ms[2 * f + o])
                       for f in range(len(lenssim.BATCH_FORMS)) for o in range(2)}}

    def batched():
        rc = L.lens_sim_image(sim.h, arr, n_sys, ptrs, sp)
        if rc:
            raise lenssim.LensSimError(rc, sim.last_error())

    batched()  # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    batched()
    e1.record(st)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1000.0
    one = [ctypes.c_void_p(o.data_ptr()) for o in outs]
    t0 = time.perf_counter()
    for i in range(n_sys):
        rc = L.lens_sim_image(sim.h, ctypes.byref(arr[i]), 1, ctypes.byref(one[i]), sp)
        if rc:
            raise lenssim.LensSimError(rc, sim.last_error())
        st.synchronize()
    t_plain = time.perf_counter() - t0
    out = {"systems": n_sys, "images_per_s": n_sys / t_batch, "plain_images_per_s": n_sys / t_plain,
           "speedup_vs_plain": t_plain / t_batch, "pairs_per_s": pairs / t_batch,
           "plain_pairs_per_s": pairs / t_plain, "batch_s": t_batch, "plain_s": t_plain, "schedule": schedule,
           "workload": ("grids 64^2, s in {1,2,3}, subhalos log-uniform in [0,100], PSF 5..31" if small else
                        "grids {64,100,128,200,256}^2, s in {1,2,3}, subhalos log-uniform in [0,20000], PSF 5..31")
                       + "; one graph launch vs per-image calls with a sync each"}
    if single_pairs_per_s > 0:
        ceiling = n_sys * single_pairs_per_s / pairs
        out["pair_rate_ceiling"] = {"images_per_s": ceiling, "speedup_vs_plain": ceiling * t_plain / n_sys,
                                    "single_image_pairs_per_s": single_pairs_per_s}
    return out


def _rel_linf(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())


def per_config_extra(sim, lenssim, W, dev, cpu_budget_s: float = 10.0):
    """Per-configuration report: for the plain (60^2), substructure (200^2, s = 3, 10k), batched
    (uneven mix) and differentiation (100^2, 15 parameters) workloads, the GPU's error against
    the FP64 oracle beside the oracle's conditioning floor (its own error when every quantity an
    FP32 evaluation must round is rounded to FP32), and the oracle's CPU throughput on this
    host; plus the plain 60^2 image's GPU images/s (a launch-bound single-system call)."""
    import torch
    import oracle
    oracle.build()
    out = {}
    cores = oracle.nthreads()

    def gpu_img(system):
        img = sim.image(system)[0]
        torch.cuda.synchronize()
        return img.cpu().numpy()

    # C1 plain
    c1 = W.plain_system()
    ref = oracle.image(c1)
    floor = _rel_linf(oracle.image(c1, fp32=True), ref)
    t0 = time.perf_counter()
    n1 = 0
    while n1 < 3 or time.perf_counter() - t0 < min(2.0, cpu_budget_s / 4):
        oracle.image(c1)
        n1 += 1
    cpu_c1 = n1 / (time.perf_counter() - t0)
    keep = []
    cc = sim.system_struct(c1, keep)
    outd = torch.empty((60, 60), device=dev)
    import ctypes
    L = lenssim.lib()
    ptr = (ctypes.c_void_p * 1)(outd.data_ptr())
    sp = int(torch.cuda.current_stream().cuda_stream)
    for _ in range(20):
        L.lens_sim_image(sim.h, ctypes.byref(cc), 1, ptr, sp)
    torch.cuda.synchronize()
    reps = 2000
    t0 = time.perf_counter()
    for _ in range(reps):
        rc = L.lens_sim_image(sim.h, ctypes.byref(cc), 1, ptr, sp)
        if rc:
            raise lenssim.LensSimError(rc, sim.last_error())
    torch.cuda.synchronize()
    gpu_c1 = reps / (time.perf_counter() - t0)
    t0 = time.perf_counter()
    for _ in range(500):
        L.lens_sim_image(sim.h, ctypes.byref(cc), 1, ptr, sp)
        torch.cuda.synchronize()
    gpu_c1_sync = 500 / (time.perf_counter() - t0)
    out["plain"] = {"workload": "60x60 at 0.05\", s = 1, SIE + shear, Sersic, 5x5 Gaussian PSF",
                    "gpu_rel_linf": _rel_linf(gpu_img(c1), ref), "oracle_floor": floor,
                    "tolerance": max(1e-5, 2 * floor), "gpu_images_per_s": gpu_c1,
                    "gpu_images_per_s_sync_each": gpu_c1_sync,
                    "cpu_oracle": {"images_per_s": cpu_c1, "cores": cores, "sample": f"{n1} full images"}}

    # C2 substructure: the first benchmark system, whole image
    c2 = W.substructure_system(1000)
    ref = oracle.image(c2)
    floor = _rel_linf(oracle.image(c2, fp32=True), ref)
    out["substructure"] = {"workload": "200x200 at 0.04\", s = 3, EPL + shear, 10,000 TNFW, Sersic, 21x21 Moffat "
                                       "(seed 1000, whole image)",
                           "gpu_rel_linf": _rel_linf(gpu_img(c2), ref), "oracle_floor": floor,
                           "tolerance": max(1e-5, 2 * floor)}

    # C3 batched: four members of the uneven mix through one batched call, whole images; the
    # oracle's CPU rate is extrapolated from two-row bands of 64 seeded members
    mix = W.batched_systems(2024, count=64)
    order = sorted(range(len(mix)), key=lambda i: mix[i].pairs())
    pick = [order[0], order[len(order) // 4], order[len(order) // 2], order[(3 * len(order)) // 5]]
    members = [mix[i] for i in pick]
    imgs = sim.image(members)
    torch.cuda.synchronize()
    errs, floors = [], []
    for sy, im in zip(members, imgs):
        r = oracle.image(sy)
        errs.append(_rel_linf(im.cpu().numpy(), r))
        floors.append(_rel_linf(oracle.image(sy, fp32=True), r))
    t_est = 0.0
    t0 = time.perf_counter()
    for sy in mix:
        ny = sy.grid.ny
        r0 = ny // 2 - 1
        ta = time.perf_counter()
        oracle.image_rows(sy, r0, r0 + 2)
        t_rows = time.perf_counter() - ta
        ta = time.perf_counter()
        if sy.psf is not None:
            oracle.convolve(np.zeros((ny, sy.grid.nx)), sy.psf)
        t_est += t_rows * ny / 2 + (time.perf_counter() - ta)
    out["batched"] = {"workload": "uneven mix: grids {64,100,128,200,256}^2, s in {1,2,3}, 0..20,000 TNFW, PSF 5..31",
                      "members": [{"grid": m.grid.nx, "s": m.grid.s, "n_sub": m.n_sub,
                                   "psf": 0 if m.psf is None else int(m.psf.shape[0]),
                                   "gpu_rel_linf": e, "oracle_floor": f, "tolerance": max(1e-5, 2 * f)}
                                  for m, e, f in zip(members, errs, floors)],
                      "cpu_oracle": {"images_per_s": len(mix) / t_est, "cores": cores, "extrapolated": True,
                                     "sample": "two central rows of each of 64 seeded members of the mix plus "
                                               "each one's full PSF convolution, extrapolated to whole images",
                                     "seconds": time.perf_counter() - t0}}

    # C4 differentiation: likelihood + gradient at 4 of the 512 points
    pb = W.diff_problem(42)
    data = W.observe(oracle.model_image(pb.system, pb.truth), pb.sigma_bkg, pb.t_exp, 42)
    idx = [0, 131, 257, 511]
    tid = sim.register_subhalos(pb.system.subhalos)
    Lg, Gg = sim.grad(pb.system, torch.from_numpy(data).to(dev), pb.sigma_bkg, pb.t_exp,
                      torch.from_numpy(pb.points).to(dev), subhalo_table=tid)
    torch.cuda.synchronize()
    Lg, Gg = Lg.cpu().numpy()[idx], Gg.cpu().numpy()[idx]
    pts = pb.points[idx].astype(np.float64)
    Lr, Gr = oracle.loglike(pb.system, data, pb.sigma_bkg, pb.t_exp, pts)
    n_cpu = max(16, cores)
    t0 = time.perf_counter()
    oracle.loglike(pb.system, data, pb.sigma_bkg, pb.t_exp, pb.points[:n_cpu].astype(np.float64))
    t_grad = time.perf_counter() - t0
    _, Gf = oracle.loglike(pb.system, data, pb.sigma_bkg, pb.t_exp, pts, fp32=True)
    # conditioning floor per component: the rounding mode's change, or the first-order change
    # of the exact gradient under a one-ulp perturbation of each parameter, whichever is larger
    lin = np.zeros_like(Gr)
    for j in range(15):
        d = np.zeros_like(pts)
        d[:, j] = np.abs(pts[:, j]) * 2.0 ** -23
        _, Gp = oracle.loglike(pb.system, data, pb.sigma_bkg, pb.t_exp, pts + d)
        _, Gm = oracle.loglike(pb.system, data, pb.sigma_bkg, pb.t_exp, pts - d)
        lin += 0.5 * np.abs(Gp - Gm)
    floor = np.maximum(np.abs(Gf - Gr), lin)
    gmax = np.abs(Gr).max(axis=1, keepdims=True)
    scale = np.maximum(np.abs(Gr), 1e-3 * gmax)
    out["differentiation"] = {
        "workload": "100x100 at 0.05\", 13x13 Gaussian PSF, 1000 fixed TNFW, 15 parameters (points 0, 131, 257, 511)",
        "logL_rel_err_max": float(np.max(np.abs(Lg - Lr) / np.abs(Lr))),
        "grad_normwise_err_max": float(np.max(np.abs(Gg - Gr).max(axis=1) / gmax[:, 0])),
        "grad_componentwise_err_max": float(np.max(np.abs(Gg - Gr) / scale)),
        "grad_rounding_floor_componentwise_max": float(np.max(np.abs(Gf - Gr) / scale)),
        "grad_conditioning_floor_componentwise_max": float(np.max(floor / scale)),
        "grad_err_over_bound_max": float(np.max((np.abs(Gg - Gr) / scale) / np.maximum(1e-4, 2.0 * floor / scale))),
        "cpu_oracle": {"gradients_per_s": n_cpu / t_grad, "cores": cores,
                       "sample": f"{n_cpu} of the 512 points, forward-mode dual numbers (15 tangents), "
                                 f"including the 10^7-pair subhalo field"}}
    return out


def measured_hbm_gbs():
    """HBM copy bandwidth measured on GB300s (MEASURED_PEAKS.json), else a fallback figure
    from an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def conv_extra(sim, W, dev, n_img: int = 4096, size: int = 256):
    """PSF step alone on a batch larger than L2: n_img x size^2 FP32 images through
    lens_sim_convolve.  k = 5 is HBM-bound (algorithmic 8 B per pixel: one read, one write);
    k = 21 is FP32-bound (2 k^2 flops per pixel)."""
    import torch
    x = torch.rand((n_img, size, size), device=dev)
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()
    res = {}
    for k in (5, 21):
        K = W.gaussian_psf(0.1, 0.04, k) if k == 5 else W.moffat_psf(3.0, 0.12, 0.04, k)
        pid = sim.register_psf(K)
        sim.convolve(x, pid, out=y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(st)
        for _ in range(reps):
            sim.convolve(x, pid, out=y)
        e1.record(st)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0 / reps
        px = n_img * size * size
        res[f"k{k}"] = {"ms": t * 1e3, "gbs_algorithmic": 8.0 * px / t / 1e9,
                        "tflops": 2.0 * k * k * px / t / 1e12}
    peak, basis = measured_hbm_gbs()
    res["hbm_peak_gbs"] = peak
    res["hbm_peak_basis"] = basis
    res["k5_frac_of_measured_hbm"] = res["k5"]["gbs_algorithmic"] / peak
    res["k5_frac_of_nominal_hbm_7900"] = res["k5"]["gbs_algorithmic"] / 7900.0
    res["workload"] = f"{n_img} x {size}^2 FP32 images, lens_sim_convolve, inputs larger than L2"
    del x, y
    torch.cuda.empty_cache()
    return res


def fft_conv_extra(sim, W, dev, n_img: int = 64):
    """FFT against direct PSF step for large kernels (the paper's 180x180 grids with kernels up
    to 135): a stack of n_img images per call through lens_sim_convolve, each method forced."""
    import torch
    st = torch.cuda.current_stream()
    res = {}
    for size, k in ((180, 135), (200, 135), (200, 75), (200, 45), (256, 101)):
        x = torch.rand((n_img, size, size), device=dev)
        y = torch.empty_like(x)
        pid = sim.register_psf(W.moffat_psf(3.0, 0.12 * k / 21.0, 0.04, k))
        row = {}
        for m in ("direct", "fft"):
            sim.set_conv_method(m)
            sim.convolve(x, pid, out=y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            e0.record(st)
            for _ in range(reps):
                sim.convolve(x, pid, out=y)
            e1.record(st)
            torch.cuda.synchronize()
            row[f"{m}_ms_per_image"] = e0.elapsed_time(e1) / reps / n_img
        row["fft_speedup"] = row["direct_ms_per_image"] / row["fft_ms_per_image"]
        res[f"{size}x{size}_k{k}"] = row
        del x, y
    sim.set_conv_method("auto")
    torch.cuda.empty_cache()
    res["workload"] = f"{n_img} images per call, Moffat kernels, lens_sim_convolve with the method forced"
    return res


def far_field_extra(sim, lenssim, W, dev, reps: int = 20):
    """The optional far-field interpolation of the subhalo sum on the benchmark image (200^2,
    s = 3, 10,000 TNFW, 21x21 PSF, seed 1000): per kappa, the fraction of (unit, subhalo) pairs
    it interpolates, the whole-image error against the FP64 oracle's exact sum, and the
    device-resident images/s (trace + PSF, CUDA events, the launch variant autotuned for that
    kappa).  kappa = 0 is the exact sum the headline measures."""
    import ctypes
    import torch
    import oracle
    oracle.build()
    system = W.substructure_system(1000)
    ref = oracle.image(system)
    floor = _rel_linf(oracle.image(system, fp32=True), ref)
    # interpolated fraction: per unit (8x4 pixels at s = 3), subhalos at box distance >= kappa h
    # that the near-field test does not mark (box distance >= 7 max(tau, 1) Rs)
    cx, cy, Rs, _, rt = system.subhalos.astype(np.float64)
    tm = np.maximum(rt / Rs, 1.0)
    g = system.grid
    dp, nx, s = float(g.dpix), g.nx, g.s
    def coord(j, b):
        return (j - 0.5 * (nx - 1) + (b + 0.5) / s - 0.5) * dp
    dists, halfw = [], []
    for by in range(g.ny // 4):
        y0, y1 = coord(by * 4, 0), coord(by * 4 + 3, s - 1)
        for bx in range(nx // 8):
            x0, x1 = coord(bx * 8, 0), coord(bx * 8 + 7, s - 1)
            ddx = np.maximum(np.maximum(x0 - cx, cx - x1), 0.0)
            ddy = np.maximum(np.maximum(y0 - cy, cy - y1), 0.0)
            dists.append(np.hypot(ddx, ddy))
            halfw.append(0.5 * max(x1 - x0, y1 - y0))
    dists = np.array(dists)
    halfw = np.array(halfw)[:, None]
    marked = dists < 7.0 * tm * Rs
    L = lenssim.lib()
    st = torch.cuda.current_stream()
    out = torch.empty((g.ny, g.nx), device=dev)
    ptrs = (ctypes.c_void_p * 1)(out.data_ptr())
    keep = []
    c = sim.system_struct(system, keep, subhalos=torch.from_numpy(system.subhalos).to(dev))
    res = {}
    for kappa in (0.0, 3.0, 4.0, 6.0):
        sim.set_far_field(kappa)
        tune = sim.autotune(system, use_cache=False)
        for _ in range(3):
            L.lens_sim_image(sim.h, ctypes.byref(c), 1, ptrs, int(st.cuda_stream))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            rc = L.lens_sim_image(sim.h, ctypes.byref(c), 1, ptrs, int(st.cuda_stream))
            if rc:
                raise lenssim.LensSimError(rc, sim.last_error())
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        frac = float(((dists >= kappa * halfw) & ~marked).mean()) if kappa > 0 else 0.0
        res[f"{kappa:g}"] = {"images_per_s": 1e3 / ms, "ms_per_image": ms, "variant": tune["name"],
                             "trace_ms_by_variant": tune["ms"], "interpolated_pair_fraction": frac,
                             "rel_linf_vs_oracle": _rel_linf(out.cpu().numpy(), ref)}
    sim.set_far_field(0.0)
    return {"kappa": res, "oracle_floor": floor, "tolerance": max(1e-5, 2 * floor),
            "stated_bound_per_subhalo": {"3": 1.2e-6, "4": 1.4e-7, "6": 6e-9},
            "workload": "200x200 at 0.04\", s = 3, EPL + shear, 10,000 TNFW, Sersic, 21x21 Moffat (seed 1000); "
                        f"{reps} device-resident calls per kappa after 3 warm-up calls"}


def subhalo_scaling_extra(sim, W, dev):
    """Trace-kernel throughput against the subhalo count on the benchmark grid (200x200, s = 3):
    the pair sum should stay at a flat pairs/s once the subhalos fill the GPU."""
    import ctypes
    import torch
    from paper_2606_01547_gb300 import lenssim
    L = lenssim.lib()
    st = torch.cuda.current_stream()
    out = torch.empty((200, 200), device=dev)
    ptrs = (ctypes.c_void_p * 1)(out.data_ptr())
    res = []
    for n_sub in (1000, 3000, 10000, 30000, 100000):
        system = W.substructure_system(2000 + n_sub, n_sub=n_sub, k=0)
        keep = []
        c = sim.system_struct(system, keep, subhalos=torch.from_numpy(system.subhalos).to(dev), use_psf=False)
        reps = 3 if n_sub >= 30000 else 10
        for _ in range(2):
            L.lens_sim_image(sim.h, ctypes.byref(c), 1, ptrs, int(st.cuda_stream))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            rc = L.lens_sim_image(sim.h, ctypes.byref(c), 1, ptrs, int(st.cuda_stream))
            if rc:
                raise lenssim.LensSimError(rc, sim.last_error())
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res.append({"n_subhalos": n_sub, "ms_per_image": ms, "pairs_per_s": system.pairs() / (ms / 1e3)})
    return {"points": res, "workload": "200x200, s = 3, no PSF, seeded TNFW populations of each size"}


def grad_extra(sim, W, dev):
    """Differentiation workload: chi^2 logL + 15-parameter adjoint at 512 points (100x100, 13x13
    PSF, 1,000 fixed subhalos); the observation is this GPU path's own truth image plus noise."""
    import torch
    pb = W.diff_problem(42)
    truth_img = sim.image(pb.system)[0].cpu().numpy()
    data = torch.from_numpy(W.observe(truth_img, pb.sigma_bkg, pb.t_exp, 42)).to(dev)
    P = torch.from_numpy(pb.points).to(dev)
    tid = sim.register_subhalos(pb.system.subhalos)
    st = torch.cuda.current_stream()
    for _ in range(2):
        sim.grad(pb.system, data, pb.sigma_bkg, pb.t_exp, P, subhalo_table=tid)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(st)
    for _ in range(reps):
        sim.grad(pb.system, data, pb.sigma_bkg, pb.t_exp, P, subhalo_table=tid)
    e1.record(st)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0 / reps
    return {"points": int(P.shape[0]), "gradients_per_s": P.shape[0] / t, "ms_per_call": 1000.0 * t,
            "workload": "100x100, 13x13 Gaussian PSF, 1000 fixed TNFW, 15 parameters, 512 points"}


def fitting_extra(sim, W, dev):
    """Particle swarm fit of the differentiation workload's 15 parameters (the paper's PSO
    benchmark, here on the EPL + shear + Sersic model): 64..512 particles, 100 iterations,
    every iteration one batched likelihood call over the swarm."""
    import torch
    from paper_2606_01547_gb300 import fitting
    pb = W.diff_problem(42)
    truth_img = sim.image(pb.system)[0].cpu().numpy()
    data = torch.from_numpy(W.observe(truth_img, pb.sigma_bkg, pb.t_exp, 42)).to(dev)
    tid = sim.register_subhalos(pb.system.subhalos)
    # untimed warm-up: workspaces and the first use of the registered table
    fitting.pso_fit(sim, pb.system, data, pb.sigma_bkg, pb.t_exp, n_particles=512, iters=2, seed=0, subhalo_table=tid)
    out = []
    for n in (64, 128, 256, 512):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fitting.pso_fit(sim, pb.system, data, pb.sigma_bkg, pb.t_exp, n_particles=n, iters=100, seed=1,
                              subhalo_table=tid)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out.append({"particles": n, "iterations": 100, "seconds": t, "evaluations_per_s": res.evaluations / t,
                    "best_logL": float(res.logL[0])})
    # L-BFGS with the adjoint's gradients (through the autograd.Function) from 64 starts 2 % off
    # the truth, all starts in one batched likelihood+gradient call per function evaluation
    import numpy as np
    rng = np.random.default_rng(3)
    starts = (pb.truth[None] * (1.0 + 0.02 * rng.standard_normal((64, 15)))).astype(np.float32)
    fitting.lbfgs_fit(sim, pb.system, data, pb.sigma_bkg, pb.t_exp, starts[:4], iters=3, restarts=1,
                      subhalo_table=tid)  # untimed warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = fitting.lbfgs_fit(sim, pb.system, data, pb.sigma_bkg, pb.t_exp, starts, iters=50, restarts=4,
                            subhalo_table=tid)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    truth = torch.from_numpy(pb.truth[None]).to(dev)
    L_truth = float(sim.grad(pb.system, data, pb.sigma_bkg, pb.t_exp, truth, want_grad=False, subhalo_table=tid)[0])
    lbfgs = {"starts": 64, "seconds": t, "point_evaluations": res.evaluations,
             "point_evaluations_per_s": res.evaluations / t, "best_logL": float(res.logL.max()),
             "logL_at_truth": L_truth}
    return {"pso": out, "lbfgs": lbfgs, "workload": "100x100, 13x13 PSF, 1000 fixed TNFW, 15 free parameters"}


def serving_extra(lenssim, W, rates, seconds: float, pool_size: int = 6000, out_sets: int = 2,
                  warmup_requests: int = 6000, settle_s: float = 3.0):
    """Serving: open-loop Poisson arrivals at each rate for `seconds`, drawn from a pool of
    `pool_size` pre-generated requests of the serving mix (70 % image / 30 % likelihood +
    gradient, grids 64..256, subhalos 0..20,000, PSF 5..31) that is cycled.  One server serves
    every rate; its PSFs are registered up front, as a deployment would, and an untimed warm-up
    (the whole pool submitted back to back) lets its slots size their workspaces and capture
    their batch graphs (a warm-up of half the pool left the first rate to meet the other half's
    largest requests, and a workspace growth inside it held the client up by 85 ms); an
    unmeasured open-loop window of `settle_s` at the first rate (at most 3,000 req/s) follows (the first window after
    the warm-up saw a one-time 58 ms overshoot of the client's own sleep, in no later window),
    and each rate's statistics are reset before it starts.  Each pool entry has `out_sets` sets
    of output buffers used in turn, so a buffer set is reused only pool_size * out_sets arrivals
    later, after its previous request finished (a reuse that had to wait for it is counted in
    `blocked_reuses`); a submit refused
    with LENS_ERR_BUSY (more than max_inflight = 4096 requests admitted) counts as rejected.
    p50/p99 are the server's own submit-to-result latencies of the admitted requests.  The image
    requests of the pool are then run one by one through lens_sim_image with a synchronisation
    each: the plain per-image path on the same GPU."""
    import collections
    import torch
    pool = W.serving_stream(7, rate=1.0, duration=1.3 * pool_size)[:pool_size]
    inputs, outs = [], []
    for rq in pool:
        g = rq.system.grid
        if rq.kind == 0:
            inputs.append(())
            outs.append([(np.empty((g.ny, g.nx), np.float32),) for _ in range(out_sets)])
        else:
            p = np.array([*rq.system.deflectors[0][1], *rq.system.deflectors[1][1], *rq.system.source[1]],
                         np.float32)
            inputs.append((np.zeros((g.ny, g.nx), np.float32), p))
            outs.append([(np.empty(1, np.float32), np.empty(15, np.float32)) for _ in range(out_sets)])

    srv = lenssim.Server(device=0)
    for rq in pool:
        srv.sim.register_psf(rq.system.psf)
    # every request is marshalled before the arrivals start, so that the open-loop client does
    # no more per arrival than one submit call (a Python client that built each request on the
    # fly fell up to 90 ms behind its schedule and then submitted in bursts)
    prepared = []
    for j, rq in enumerate(pool):
        b = inputs[j]
        prepared.append([srv.prepare_image(rq.system, outs[j][c][0]) if rq.kind == 0 else
                         srv.prepare_loglike(rq.system, b[0], 0.01, 1000.0, b[1], outs[j][c][0], outs[j][c][1])
                         for c in range(out_sets)])

    def submit(srv, j, c):
        return srv.submit_prepared(prepared[j][c])
    t0 = time.perf_counter()
    n_warm = min(warmup_requests, pool_size)
    warm = collections.deque()
    for j in range(n_warm):
        if len(warm) >= 2048:  # stays below the server's max_inflight admission limit
            srv.wait(warm.popleft(), 600000)
        warm.append(submit(srv, j, 0))
    for t in warm:
        srv.wait(t, 600000)
    t_warm = time.perf_counter() - t0
    if settle_s > 0 and rates:
        settle_rate = min(rates[0], 3000.0)
        rng = np.random.default_rng(12345)
        arr = np.cumsum(rng.exponential(1.0 / settle_rate, int(settle_rate * settle_s * 1.2) + 16))
        ts0 = time.perf_counter()
        settle = {}
        for i, ta in enumerate(arr[arr < settle_s]):
            delay = ta - (time.perf_counter() - ts0)
            if delay > 0:
                time.sleep(delay)
            j = i % len(pool)
            if j in settle:  # an entry's buffers are reused only after its previous request
                srv.wait(settle.pop(j), 600000)
            try:
                settle[j] = submit(srv, j, 0)
            except lenssim.LensSimError as e:
                if e.code != lenssim.LENS_ERR_BUSY:
                    raise
        for t in settle.values():
            srv.wait(t, 600000)
    out = []
    for rate in rates:
        srv.reset_stats()
        rng = np.random.default_rng(int(rate))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, int(rate * seconds * 1.2) + 16))
        arrivals = arrivals[arrivals < seconds]
        codes = collections.Counter()
        pending = {}
        rejected = blocked = img_ok = 0
        late = 0.0
        gc.collect()
        gc.disable()  # no collector pauses inside the arrival schedule
        time.sleep(0.2)
        t0 = time.perf_counter()
        for i, ta in enumerate(arrivals):
            delay = ta - (time.perf_counter() - t0)
            if delay > 0:
                # time.sleep overshoots short delays (timer slack, ~50-80 us): at 20,000 req/s
                # (50 us between arrivals) it let the client fall up to 51 ms behind its schedule
                # and then submit in a burst; the last 0.3 ms are spun instead
                if delay > 3e-4:
                    time.sleep(delay - 3e-4)
                while time.perf_counter() - t0 < ta:
                    pass
            else:
                late = max(late, -delay)
            j = i % len(pool)
            c = (i // len(pool)) % out_sets
            prev = pending.pop((j, c), None)
            if prev is not None:
                rc = srv.poll(prev)
                if rc == lenssim.LENS_ERR_BUSY:
                    blocked += 1
                    rc = srv.wait(prev, 600000)
                codes[rc] += 1
                img_ok += int(rc == 0 and pool[j].kind == 0)
            try:
                pending[(j, c)] = submit(srv, j, c)
            except lenssim.LensSimError as e:
                if e.code != lenssim.LENS_ERR_BUSY:
                    raise
                rejected += 1
        t_submit = time.perf_counter() - t0
        for (jj, _), t in pending.items():
            rc = srv.wait(t, 600000)
            codes[rc] += 1
            img_ok += int(rc == 0 and pool[jj].kind == 0)
        t_all = time.perf_counter() - t0
        gc.enable()
        st = srv.stats()
        rec = {"rate_req_per_s": rate, "seconds": seconds, "offered": int(len(arrivals)),
               "submit_seconds": t_submit, "max_submit_lag_s": late, "rejected_busy": rejected,
               "blocked_reuses": blocked, "admitted": int(sum(codes.values())), "completed_ok": codes.get(0, 0),
               "failed": {str(k): v for k, v in codes.items() if k != 0},
               "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "served_req_per_s": st["requests_per_s"],
               "images_completed": img_ok,
               "served_images_per_s": st["requests_per_s"] * img_ok / max(1, codes.get(0, 0)),
               "completed_per_wall_s": codes.get(0, 0) / t_all}
        if rec["failed"]:
            rec["last_error"] = srv.last_error()
        out.append(rec)
    srv.close()
    sim = lenssim.Simulator(device=0)
    imgs = [rq.system for rq in pool if rq.kind == 0][:2000]
    dev_out = [torch.empty((s_.grid.ny, s_.grid.nx), device="cuda") for s_ in imgs]
    for s_, o in zip(imgs[:50], dev_out):  # untimed: workspaces and PSF registrations
        sim.image(s_, out=[o])
    for s_ in imgs:
        sim.register_psf(s_.psf)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for s_, o in zip(imgs, dev_out):
        sim.image(s_, out=[o])
        torch.cuda.synchronize()
    plain = len(imgs) / (time.perf_counter() - t1)
    sim.close()
    return {"rates": out, "pool": pool_size, "warmup_requests": n_warm, "warmup_seconds": t_warm,
            "settle_seconds": settle_s,
            "plain_images_per_s": plain, "plain_images": len(imgs),
            "mix": "70% image / 30% likelihood+gradient, grids 64..256 (even), s = 1, subhalos log-uniform "
                   "0..20000, PSF 5..31"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--clock-soak-s", type=float, default=1.5,
                    help="seconds of untimed repeats of the step during which clocks are sampled as well")
    ap.add_argument("--ref-budget-s", type=float, default=90.0,
                    help="reference arm: seconds of oracle work for the whole run, split over its steps")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched, gradient and serving lines")
    ap.add_argument("--variant", type=int, default=-1, help="fixed trace launch variant instead of autotuning")
    ap.add_argument("--far-field", type=float, default=0.0, metavar="KAPPA",
                    help="time the optional far-field interpolation of the subhalo sum (approximate; "
                         "0 = the exact sum, the headline)")
    ap.add_argument("--extra-only", default="", choices=["", "differentiation", "batched", "batched_small_systems",
                                                          "fitting", "scaling", "far_field", "serving", "per_config"],
                    help="profiling mode: only this one extra measurement")
    ap.add_argument("--fft-only", type=int, default=0, metavar="N_IMG",
                    help="profiling mode: only the FFT-versus-direct PSF measurement (N_IMG images per call)")
    ap.add_argument("--psf-only", type=int, default=0, metavar="N_IMG",
                    help="only the standalone PSF measurement on N_IMG 256^2 images (profiling runs)")
    ap.add_argument("--batch-systems", type=int, default=4096)
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[100.0, 1000.0, 3000.0, 10000.0, 20000.0, 30000.0])
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.extra_only:
        import torch
        from paper_2606_01547_gb300 import lenssim
        from paper_2606_01547_gb300 import workloads as W
        dev = torch.device("cuda", 0)
        sim = lenssim.Simulator(device=0)
        fn = {"differentiation": lambda: grad_extra(sim, W, dev),
              "batched": lambda: batched_extra(sim, lenssim, W, dev, args.batch_systems),
              "batched_small_systems": lambda: batched_extra(sim, lenssim, W, dev, args.batch_systems, small=True),
              "fitting": lambda: fitting_extra(sim, W, dev),
              "scaling": lambda: subhalo_scaling_extra(sim, W, dev),
              "far_field": lambda: far_field_extra(sim, lenssim, W, dev),
              "serving": lambda: serving_extra(lenssim, W, args.serve_rates, args.serve_seconds),
              "per_config": lambda: per_config_extra(sim, lenssim, W, dev, args.cpu_budget_s)}[args.extra_only]
        print(json.dumps({args.extra_only: fn()}), flush=True)
        sim.close()
        return
    if args.fft_only:
        import torch
        from paper_2606_01547_gb300 import lenssim
        from paper_2606_01547_gb300 import workloads as W
        sim = lenssim.Simulator(device=0)
        print(json.dumps({"psf_fft": fft_conv_extra(sim, W, torch.device("cuda", 0), n_img=args.fft_only)}), flush=True)
        sim.close()
        return
    if args.psf_only:
        import torch
        from paper_2606_01547_gb300 import lenssim
        from paper_2606_01547_gb300 import workloads as W
        sim = lenssim.Simulator(device=0)
        print(json.dumps({"psf_conv": conv_extra(sim, W, torch.device("cuda", 0), n_img=args.psf_only)}), flush=True)
        sim.close()
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
