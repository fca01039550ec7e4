#!/usr/bin/env python
"""Throughput of the q-LSKUM hot path on GB300: point-iterations per second.

One step = one pseudo-time iteration of Algorithm 1 over the whole cloud
(second-order q-LSKUM, 3 inner iterations, RK4 = 4 residual evaluations, each
q-derivatives + fused flux residual/update) on a seeded synthetic NACA 0012
cloud of 2,498,560 points at M = 1.2, alpha = 0. Inputs are resident in HBM
when the timed region starts; the working set (~3 GB) is far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, torchrun), weak scaling.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "q-LSKUM point-iterations/s at 2.5M pts (FP64 vs mixed); % of HBM roofline"
UNIT = "point-iterations/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="naca0012_2p5m")
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--inner", type=int, default=3)
    ap.add_argument("--scheme", choices=["euler", "rk4"], default="rk4")
    ap.add_argument("--mach", type=float, default=1.2)
    ap.add_argument("--aoa", type=float, default=0.0)
    ap.add_argument("--cfl", type=float, default=0.2)
    ap.add_argument("--limiter", type=float, default=1.0, help="Venkatakrishnan K (0: none)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--reorder", type=int, default=1, help="0 input order, 1 Morton, 2 reverse Cuthill-McKee")
    ap.add_argument("--shuffle", type=int, default=1, help="present the cloud in random point order")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ref-extra", dest="ref_extra", action="store_false",
                    help="reference arm: skip the serial and all-core 160k-point oracle runs")
    ap.add_argument("--single-form", action="store_true", help="time only --precision's form")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solves form")
    ap.add_argument("--no-error", action="store_true", help="skip the mixed form's error against FP64")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint form")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the forward-Euler, input-order and 10M-point forms")
    ap.add_argument("--tuning", default="auto",
                    help="mixed launch shapes: 'auto' (autotune on the cloud) or 'F,Q' (flux, q-derivative variant)")
    ap.add_argument("--residuals-only", type=int, default=0, metavar="N",
                    help="no timing: create the configured form (--precision, --tuning), set the timed start "
                         "state and evaluate the residual N times (a short program for ncu captures)")
    ap.add_argument("--accuracy", action="store_true",
                    help="instead of timing: the mixed form's converged error against FP64 at 160k and 2.5M points")
    ap.add_argument("--acc-iters-160k", type=int, default=60000)
    ap.add_argument("--acc-cfl-160k", type=float, default=1.0)
    ap.add_argument("--acc-iters-2p5m", type=int, default=300000)
    ap.add_argument("--acc-cfl-2p5m", type=float, default=0.5, help="CFL 0.8 loses positivity on this cloud")
    ap.add_argument("--acc-iters-fp64-restart", type=int, default=10000,
                    help="2.5M: iterations both forms run on from the mixed form's state")
    ap.add_argument("--acc-chunk", type=int, default=2500)
    ap.add_argument("--batch-clouds", type=int, default=16)
    ap.add_argument("--batch-conditions", type=int, default=3)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = sorted(float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit())
        smax = max((float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(self.rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def algorithmic_bytes_per_point(kernel, dbar, order, scheme, stage_avg=True):
    """Bytes each array contributes once per launch, per point (FP64 layout):
    q 32, q-derivatives 64, coordinates 16, normals 16, flag 1, dmin 8, CSR
    offset 4, and per edge: index 4, mask 1, LS weights 16 (fused kernel:
    flux weights 16), half offsets (P_i - P_0)/2 16 (second order).
    Neighbour gathers are assumed served from cache."""
    if kernel == "flux":
        b = 32 + 16 + 16 + 1 + 4 + dbar * (4 + 1 + 16)       # q, xy, nrm, flag, off, edges
        if order == 2:
            b += 64 + dbar * 16                               # own q-derivatives, half offsets
        b += 32 + 32 + 32                                     # U^n read, U_out and q_out written
        if scheme == "rk4":
            # dt (+dmin) at stage 0, acc written at 0-2, read at 1-3
            b += (8 + 8 + 3 * 8 + 3 * 32 + 3 * 32) / 4.0 if stage_avg else 0
        else:
            b += 16
        return b
    if kernel == "qgrad_first":
        return 32 + 4 + dbar * (4 + 16) + 64
    if kernel == "qgrad_inner":
        # first-order result G1 64, previous iterate 64, offset 4, per edge
        # index 4 + weights 16 + half offset 16, new iterate 64 (no q)
        return 64 + 64 + 4 + dbar * (4 + 16 + 16) + 64
    if kernel == "qgrad_limit_extra":
        # per stage with the limiter after inner passes: the extremum
        # measure written by the first pass and read by the last, dmin
        return 32 + 32 + 8
    raise ValueError(kernel)


def algorithmic_bytes_per_point_mixed(kernel, dbar, order, scheme):
    """Mixed layout, bytes each array contributes once per launch, per point.
    Flux: q 16 (FP32), normal 8, flag 1, CSR offset 4, U^n 32 and U_out 32
    (FP64), q_out 16, own q-derivatives 32 (order 2), per SELL slot the index
    word (with the sub-stencil bits) 4 + (dx, dy, w_s, w_n) 16; RK4 terms
    averaged over the 4 stages: dt written (FP64) and dmin read (FP32) at
    stage 0, dt read at stages 1-3, the FP32 accumulator written at 0-2 and
    read at 1-3. q-derivative pass: own q 16, CSR offset 4, per slot the
    index word 4 + (a_x, a_y) 8, the new derivatives 32; an inner pass reads
    the first pass's result 32 instead of q, its own previous derivatives 32
    and the normal matrix (Sxx, Sxy, Syy) 16 from which the slot offsets are
    recovered; with the limiter after inner passes, the first pass writes the
    extremum measure 16 and the last reads it with dmin 4. Neighbour gathers
    are served from cache."""
    if kernel == "flux":
        b = 16 + 8 + 1 + 4 + 32 + 32 + 16 + dbar * 20
        if order == 2:
            b += 32
        if scheme == "rk4":
            b += (8 + 4 + 3 * 8 + 3 * 16 + 3 * 16) / 4.0
        else:
            b += 8 + 4
        return b
    if kernel == "qgrad_first":
        return 16 + 4 + dbar * 12 + 32
    if kernel == "qgrad_inner":
        return 32 + 32 + 16 + 4 + dbar * 12 + 32
    if kernel == "qgrad_limit_extra":
        return 16 + 16 + 4
    raise ValueError(kernel)


# Per-unit figures of the FP64 fused flux kernel (ncu counters, 640k-point
# capture, profiles/k_flux_update_fp64_naca0012_640k.md): executed FP64
# instructions per stencil edge (every FP64 instruction, of which DFMA + DMUL +
# DADD are 176.0) and the flops they carry (2 DFMA + DMUL + DADD); DRAM bytes
# per point of one full-size 2.5M launch (single-pass capture,
# profiles/launch_list_naca0012_2p5m_fp64.md).
FP64_INSTR_PER_EDGE_FLUX = 178.34
FP64_FLOPS_PER_EDGE_FLUX = 285.05
FLUX_DRAM_BYTES_PER_POINT = 598.0
# FP64 peak: ncu's DFMA unit count, 304 FP64 thread-instructions per cycle
# (each DFMA 2 flops), at the 2070 MHz maximum SM clock
FP64_PEAK_GINSTR = 304 * 2.070
FP64_PEAK_GFLOPS = 2 * FP64_PEAK_GINSTR


def roofline_fp64(flux_avg_s, n, dbar, fb, achieved_gbs, peaks, peak_src, fp64_measured=None):
    """The FP64 flux kernel is bound by the FP64 pipe: its issue rate of FP64
    instructions (a DMUL or DADD takes a slot as a DFMA does) against the
    pipe's 304 per cycle; the same rate against the FP64 multiply-add rate
    measured on this GPU (lskum_probe_peak, GFLOP/s / 2); the flop rate and
    the HBM view beside it, the latter also as flat keys."""
    instr = FP64_INSTR_PER_EDGE_FLUX * dbar * n
    flops = FP64_FLOPS_PER_EDGE_FLUX * dbar * n
    achieved = instr / flux_avg_s / 1e9
    gflops = flops / flux_avg_s / 1e9
    r = {"bound": "alu", "kernel": "k_flux_update", "achieved": achieved,
         "peak": FP64_PEAK_GINSTR, "unit": "G FP64 instructions/s", "frac": achieved / FP64_PEAK_GINSTR,
         "traffic": FLUX_DRAM_BYTES_PER_POINT * n,
         "fp64_instructions_per_launch": instr, "flops_per_launch": flops,
         "gflops": gflops, "gflops_peak": FP64_PEAK_GFLOPS, "gflops_frac": gflops / FP64_PEAK_GFLOPS,
         "avg_launch_ms": flux_avg_s * 1e3,
         "peak_source": "derived: 304 FP64 instructions/cycle x 2.07 GHz (ncu unit count, max SM clock)",
         "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
         "hbm_frac": achieved_gbs / peaks["hbm_gbs"], "hbm_algorithmic_bytes_per_launch": fb,
         "hbm_traffic_bytes_per_launch": FLUX_DRAM_BYTES_PER_POINT * n, "hbm_peak_source": peak_src,
         "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": achieved_gbs / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": fb,
                 "peak_source": peak_src}}
    if fp64_measured:
        r["fp64_fma_measured_gflops"] = fp64_measured
        r["frac_of_measured_fma_rate"] = achieved / (fp64_measured / 2.0)
        r["gflops_frac_of_measured"] = gflops / fp64_measured
    return r


# ----------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# ----------------------------------------------------------------------------
def host_cpu():
    """(logical CPUs this process may use, CPU model name)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        cores = os.cpu_count() or 1
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
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return cores, model or platform.machine()


def oracle_iterations(cloud, mask, U, args, iters, threads):
    """Time `iters` single iterations of the oracle's solver loop (timestep,
    the scheme's residual evaluations, the update, the residue) on `threads`
    host threads; returns the per-iteration wall times and the final state."""
    import oracle
    oracle.set_threads(threads)
    scheme = 1 if args.scheme == "rk4" else 0
    times = []
    for _ in range(iters):
        t0 = time.perf_counter()
        U, _ = oracle.solve(cloud, mask, U, 1, order=args.order, inner=args.inner, scheme=scheme, cfl=args.cfl,
                            mach=args.mach, aoa_deg=args.aoa, limiter=args.limiter)
        times.append(time.perf_counter() - t0)
    return times, U


def run_reference(args, rank, world):
    """The FP64 CPU oracle on this host's cores, on the whole configured
    cloud: every step is one full iteration of the oracle's solver loop,
    with the points of each pass shared out among all host threads (its
    OpenMP build, bitwise the serial one). Also reported: the serial oracle
    and the all-core oracle on the 160k-point cloud (median of 3 runs each)."""
    if rank != 0:
        return 0
    import statistics

    import oracle
    from paper_2403_13287_gb300.cloudgen import CLOUDS, naca0012_cloud, smooth_state

    cores, model = host_cpu()
    W, L = CLOUDS[args.workload]
    cloud = naca0012_cloud(W, L, shuffle=bool(args.shuffle))
    n = cloud["n"]
    mask = oracle.split_stencils(cloud)
    U = smooth_state(cloud, args.mach, args.aoa, amp=0.05, seed=7)
    threads = oracle.set_threads(cores)
    _, U = oracle_iterations(cloud, mask, U, args, args.warmup, threads)
    t0 = time.perf_counter()
    times, U = oracle_iterations(cloud, mask, U, args, args.steps, threads)
    total = time.perf_counter() - t0
    value = n * args.steps / total
    # the 160k-point cloud: serial and all cores, 10 iterations each, median of 3
    extra = {}
    W2, L2 = CLOUDS["naca0012_160k"]
    c2 = naca0012_cloud(W2, L2, shuffle=bool(args.shuffle)) if args.ref_extra else None
    m2 = oracle.split_stencils(c2) if c2 else None
    U2 = smooth_state(c2, args.mach, args.aoa, amp=0.05, seed=7) if c2 else None
    for key, thr, its in ((("serial_160k", 1, 10), ("all_cores_160k", threads, 10)) if c2 else ()):
        runs = []
        for _ in range(3):
            ts, _ = oracle_iterations(c2, m2, U2, args, its, thr)
            runs.append(c2["n"] * its / sum(ts))
        extra[key] = {"value": statistics.median(runs), "unit": UNIT, "threads": thr, "iterations": its,
                      "runs": runs, "points": int(c2["n"]), "rdp_s": 1.0 / statistics.median(runs)}
    oracle.set_threads(1)
    sample = ("the whole %d-point cloud, one full %s iteration of the oracle's solver loop per step "
              "(timestep, %d residual evaluations with q_derivatives (%d inner iterations) and "
              "flux_residual, the update, the residue) on %d host threads (OpenMP over points, bitwise "
              "the serial oracle); %s" % (n, args.scheme.upper(), 4 if args.scheme == "rk4" else 1, args.inner,
                                          threads, model))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": args.workload, "points": n, "order": args.order,
                   "inner_iters": args.inner, "limiter_K": args.limiter, "scheme": args.scheme, "mach": args.mach,
                   "aoa_deg": args.aoa, "cfl": args.cfl},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "nproc": cores, "cpu_model": model,
                         "ms_per_iteration_median": 1e3 * statistics.median(times)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "rdp_s": 1.0 / value,
        "oracle_160k": extra,
    }
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(value, dist):
    """The largest of every rank's value (the slowest replica's time); the
    value itself without a process group."""
    if not dist:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(points, steps, ms, world):
    """Whole-job point-iterations/s of `world` replicas that each advanced
    `points` points by `steps` iterations, the slowest taking `ms`."""
    return world * points * steps / (ms / 1e3)


def cpu_baseline_sample(cloud, mask, args):
    """The oracle as it stands on all host cores (its OpenMP build, bitwise
    the serial one): one full iteration of its solver loop over the whole
    cloud from the timed form's start state."""
    from paper_2403_13287_gb300.cloudgen import smooth_state
    cores, model = host_cpu()
    U = smooth_state(cloud, args.mach, args.aoa, amp=0.05, seed=7)
    import oracle
    threads = oracle.set_threads(cores)
    times, _ = oracle_iterations(cloud, mask, U, args, 1, threads)
    oracle.set_threads(1)
    return {"value": cloud["n"] / times[0], "unit": UNIT, "cores": threads, "kind": "oracle",
            "nproc": cores, "cpu_model": model,
            "sample": "one full %s iteration of the oracle's solver loop over all %d points (%.1f s) on %d host "
                      "threads" % (args.scheme.upper(), cloud["n"], times[0], threads)}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def measure_form(args, cloud, precision, dist, sampler):
    """Create a solver in one precision, warm up, time args.steps iterations
    with CUDA events on the library's stream (barrier + synchronize on both
    sides), and read the per-kernel event times."""
    import torch

    from paper_2403_13287_gb300 import lskum

    scheme = 1 if args.scheme == "rk4" else 0
    stream = torch.cuda.current_stream()
    solver = lskum.Solver(cloud, order=args.order, inner_iters=args.inner, time_scheme=scheme,
                          cfl=args.cfl, mach=args.mach, aoa_deg=args.aoa, reorder=args.reorder,
                          limiter_K=args.limiter, precision=1 if precision == "mixed" else 0,
                          stream=stream.cuda_stream, boundary=getattr(args, "boundary", 0))
    # start from a developed-looking, non-uniform state: after an impulsive
    # start most of the cloud is still exactly uniform, where a perturbation
    # dG vanishes identically, and a few iterations would not be representative
    from paper_2403_13287_gb300.cloudgen import smooth_state
    solver.set_state(smooth_state(cloud, args.mach, args.aoa, amp=0.05, seed=7))
    # the mixed kernels come in several launch shapes: pick them on this cloud
    tuning = None
    if precision == "mixed":
        if args.tuning == "auto":
            tuning = solver.autotune(reps=5)
        else:
            fv, qv = (int(v) for v in args.tuning.split(","))
            solver.set_tuning(fv, qv)
            tuning = {"flux_variant": fv, "qgrad_variant": qv, "fixed": True}
    solver.step(args.warmup, history=False)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    solver.profile(True)
    launches0 = solver.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solver.step(args.steps, history=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = solver.launch_count() - launches0
    flux_ms, flux_n = solver.kernel_time(lskum.LSKUM_KERNEL_FLUX)
    qg_ms, qg_n = solver.kernel_time(lskum.LSKUM_KERNEL_QGRAD)
    solver.profile(False)
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ms, dist)
    return {"solver": solver, "ms": ms, "launches": launches, "flux_ms": flux_ms, "flux_n": flux_n,
            "qg_ms": qg_ms, "qg_n": qg_n, "clocks": clocks, "tuning": tuning}


def measure_e2e(solver, n, steps, dist):
    """Same metric through the public API with host buffers: per step the
    state goes host -> device, one iteration runs, the state and the residue
    come back to pinned host memory."""
    import torch
    Uh = torch.empty((4, n), dtype=torch.float64, pin_memory=True).numpy()
    Uh[...] = solver.get_state()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        solver.set_state(Uh)
        solver.step(1, history=True)
        solver.get_state(out=Uh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    return n * steps / e2e_s


# DRAM bytes per point of one launch of the mixed kernels on the 2.5M-point
# workload, from a full-size single-pass ncu capture of the current kernels
# (profiles/mixed_kernels_naca0012_2p5m.md); None where not captured
MIXED_TRAFFIC_PER_POINT = {"flux": 345.9, "qgrad": 193.2}
# warp instructions per stencil edge of the mixed flux kernel at its autotuned
# shape (64 x 12; ncu smsp__inst_executed.sum, 640k-point capture with
# 5,167,022 edges, profiles/k_flux_update_mixed_naca0012_640k.md), for the
# issue view: 4 warp instructions per cycle per SM at the 2.07 GHz maximum
# SM clock
MIXED_FLUX_WARP_INSTR_PER_EDGE = 55941364 / 5167022
ISSUE_PEAK_GINSTR = 152 * 4 * 2.070


def form_summary(args, r, n, dbar, world, precision, peaks, peak_src, probes=None):
    flux_avg_s = (r["flux_ms"] / max(r["flux_n"], 1)) / 1e3
    if precision == "mixed":
        fb = algorithmic_bytes_per_point_mixed("flux", dbar, args.order, args.scheme) * n
        gbs = fb / flux_avg_s / 1e9
        tf = MIXED_TRAFFIC_PER_POINT["flux"]
        flux_roof = {"bound": "hbm", "kernel": "k_flux_update_mixed", "achieved": gbs,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                     "traffic": tf * n if tf else None, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": fb, "avg_launch_ms": flux_avg_s * 1e3,
                     "share_of_kernel_time": r["flux_ms"] / (r["flux_ms"] + r["qg_ms"])}
        # the issue view: warp instructions per launch over the duration
        wi = MIXED_FLUX_WARP_INSTR_PER_EDGE * dbar * n
        flux_roof["issue"] = {"achieved": wi / flux_avg_s / 1e9, "peak": ISSUE_PEAK_GINSTR,
                              "unit": "G warp instructions/s",
                              "frac": wi / flux_avg_s / 1e9 / ISSUE_PEAK_GINSTR,
                              "warp_instructions_per_launch": wi,
                              "peak_source": "derived: 4 warp instructions/cycle/SM x 152 SMs x 2.07 GHz"}
        roofline = flux_roof
        if r["qg_n"]:
            # launches per stage: one first-order pass, then the inner passes
            per_stage = args.inner + 1
            qb = (algorithmic_bytes_per_point_mixed("qgrad_first", dbar, args.order, args.scheme)
                  + args.inner * algorithmic_bytes_per_point_mixed("qgrad_inner", dbar, args.order, args.scheme)
                  + (algorithmic_bytes_per_point_mixed("qgrad_limit_extra", dbar, args.order, args.scheme)
                     if args.limiter > 0 and args.inner > 0 else 0.0)
                  ) / per_stage * n
            qg_avg_s = (r["qg_ms"] / r["qg_n"]) / 1e3
            qgbs = qb / qg_avg_s / 1e9
            tq = MIXED_TRAFFIC_PER_POINT["qgrad"]
            qg_roof = {"bound": "hbm", "kernel": "k_qgrad_mixed", "achieved": qgbs, "peak": peaks["hbm_gbs"],
                       "unit": "GB/s", "frac": qgbs / peaks["hbm_gbs"], "traffic": tq * n if tq else None,
                       "peak_source": peak_src, "algorithmic_bytes_per_launch": qb,
                       "avg_launch_ms": qg_avg_s * 1e3,
                       "share_of_kernel_time": r["qg_ms"] / (r["flux_ms"] + r["qg_ms"])}
            # the roofline line names the kernel that takes most of the step
            if r["qg_ms"] > r["flux_ms"]:
                roofline = dict(qg_roof, other=flux_roof)
            else:
                roofline = dict(flux_roof, other=qg_roof)
    else:
        fb = algorithmic_bytes_per_point("flux", dbar, args.order, args.scheme) * n
        gbs = fb / flux_avg_s / 1e9
        roofline = roofline_fp64(flux_avg_s, n, dbar, fb, gbs, peaks, peak_src,
                                 (probes or {}).get("fp64_fma_gflops"))
    value = replicas_value(n, args.steps, r["ms"], world)
    return {"value": value, "edge_iterations_per_s": value * dbar, "ms_per_step": r["ms"] / args.steps,
            "dtype": "f32/f64 mixed" if precision == "mixed" else "f64", "roofline": roofline,
            "kernels": {"k_flux_update": {"launches": r["flux_n"], "total_ms": r["flux_ms"]},
                        "k_qgrad": {"launches": r["qg_n"], "total_ms": r["qg_ms"]}},
            "gpu_launches": r["launches"]}


def rel(a, b, scale=None):
    s = abs(b) if scale is None else abs(scale)
    return abs(a - b) / s if s > 0 else None


def compare_forms(cloud, mach, aoa, cfl, limiter, iters, order, inner, tuning, U0, stream):
    """The mixed form against the FP64 form from the same start state after
    `iters` iterations: Cl, Cd (relative; at alpha = 0, Cl against |Cd|), the
    wall Cp, the residue histories and the states; and the residual of both
    forms at the FP64 end state."""
    import numpy as np
    import torch

    from paper_2403_13287_gb300 import lskum
    out = {}
    res = {}
    for prec in (0, 1):
        s = lskum.Solver(cloud, order=order, inner_iters=inner, time_scheme=1, cfl=cfl, mach=mach, aoa_deg=aoa,
                         reorder=1, limiter_K=limiter, precision=prec, stream=stream)
        if prec == 1 and tuning:
            s.set_tuning(tuning["flux_variant"], tuning["qgrad_variant"])
        if U0 is not None:
            s.set_state(U0)
        h = s.step(iters)
        cl, cd, cp = s.forces()
        res[prec] = {"solver": s, "hist": h, "cl": cl, "cd": cd, "cp": cp, "U": s.get_state()}
    f, m = res[0], res[1]
    Ud = torch.from_numpy(f["U"]).cuda()
    R64 = f["solver"].residual(Ud).cpu().numpy()
    Rm = m["solver"].residual(Ud).cpu().numpy()
    for r in res.values():
        r["solver"].close()
    # at alpha = 0 the lift vanishes by symmetry (up to the cloud's jitter):
    # its error is measured against |Cd|
    small_cl = aoa == 0.0
    h64, hm = f["hist"], m["hist"]
    # the residue histories are compared while the FP64 residue is above the
    # mixed form's FP32 floor (1e-4 of its maximum)
    live = h64 > 1e-4 * h64.max()
    live[0] = False
    out.update({
        "iterations": iters, "cl_fp64": f["cl"], "cd_fp64": f["cd"], "cl_mixed": m["cl"], "cd_mixed": m["cd"],
        "cl_rel_err": rel(m["cl"], f["cl"], f["cd"] if small_cl else None),
        "cl_err_scale": "|Cd| (Cl ~ 0)" if small_cl else "|Cl|",
        "cd_rel_err": rel(m["cd"], f["cd"]),
        "cp_max_abs_err": float(np.max(np.abs(m["cp"] - f["cp"]))),
        "residue_history_max_rel_gap": float(np.max(np.abs(hm[live] - h64[live]) / h64[live])),
        "residue_history_compared_iterations": int(live.sum()),
        "residue_last_fp64": float(h64[-1]), "residue_last_mixed": float(hm[-1]),
        "residue_drop_fp64": float(h64[-1] / h64.max()), "residue_drop_mixed": float(hm[-1] / hm.max()),
        "state_max_rel_err": float(np.max(np.abs(m["U"] - f["U"]) / (np.abs(f["U"]) + 1e-3))),
        "residual_at_fp64_state": {"max_abs_err_over_max_abs": float(np.abs(Rm - R64).max() / np.abs(R64).max()),
                                   "rel_l2": float(np.linalg.norm(Rm - R64) / np.linalg.norm(R64))},
    })
    return out


def summary_of(line, forms):
    """The headline figures of every form in a few flat keys (printed last on
    the line, so a truncated tail still shows them)."""
    out = {"value": line["value"], "rdp_s": 1.0 / line["value"],
           "edge_iterations_per_s": line.get("edge_iterations_per_s"),
           "roofline_frac": line["roofline"].get("frac"), "roofline_hbm_frac": line["roofline"].get("hbm_frac")}
    for k in ("fp64", "mixed"):
        f = forms.get(k)
        if f:
            out[k + "_value"] = f["value"]
            out[k + "_ms_per_step"] = f["ms_per_step"]
    mx = forms.get("mixed")
    if mx:
        ro = mx["roofline"]
        fl = ro if ro.get("kernel") == "k_flux_update_mixed" else ro.get("other", {})
        qg = ro if ro.get("kernel") == "k_qgrad_mixed" else ro.get("other", {})
        out["mixed_flux_hbm_frac"] = fl.get("frac")
        out["mixed_flux_ms_per_launch"] = fl.get("avg_launch_ms")
        out["mixed_qgrad_hbm_frac"] = qg.get("frac")
        err = mx.get("error")
        if err:
            c = err["converged_10k"]
            out["mixed_converged_cl_rel_err"] = c["cl_rel_err"]
            out["mixed_converged_cd_rel_err"] = c["cd_rel_err"]
            out["mixed_converged_cp_max_abs_err"] = c["cp_max_abs_err"]
            b = err["bench_cloud_after_timed_steps"]
            out["mixed_residual_rel_l2_err"] = b["residual_at_fp64_state"]["rel_l2"]
            out["mixed_cd_rel_err_after_timed_steps"] = b["cd_rel_err"]
    for k in ("mixed_speedup_vs_fp64", "batched_speedup_vs_fp64"):
        if k in forms:
            out[k] = forms[k]
    if "batched" in forms:
        out["batched_value"] = forms["batched"]["value"]
        out["batched_speedup_vs_sequential"] = forms["batched"]["speedup_vs_sequential"]
    if "mixed_10m" in forms:
        out["mixed_10m_value"] = forms["mixed_10m"]["value"]
    cb = line.get("cpu_baseline")
    if cb:
        out["cpu_baseline_value"] = cb["value"]
        out["cpu_baseline_cores"] = cb["cores"]
    return out


def measure_mixed_error(args, cloud, tuning, stream):
    """The error of the mixed form beside its speedup: on the bench cloud
    after the warm-up plus timed iterations from the timed start state, and
    on a 10k-point cloud under the same conditions (CFL 1.5) run until the
    residue has fallen by more than eight decades (converged Cl, Cd, Cp)."""
    from paper_2403_13287_gb300.cloudgen import naca0012_cloud, smooth_state
    U0 = smooth_state(cloud, args.mach, args.aoa, amp=0.05, seed=7)
    short = compare_forms(cloud, args.mach, args.aoa, args.cfl, args.limiter, args.warmup + args.steps,
                          args.order, args.inner, tuning, U0, stream)
    small = naca0012_cloud(128, 77, seed=11)
    conv = compare_forms(small, args.mach, args.aoa, 1.5, args.limiter, 12000, args.order, args.inner, None,
                         None, stream)
    conv["cloud"] = "naca0012 128x77 (9,984 points), seed 11, from the free stream, CFL 1.5"
    return {"bench_cloud_after_timed_steps": short, "converged_10k": conv}


def converge(solver, iters, chunk):
    """Step `solver` `iters` iterations in chunks; the residue history and
    (iteration, Cl, Cd) after every chunk."""
    import numpy as np
    hist, forces = [], []
    done = 0
    while done < iters:
        h = solver.step(min(chunk, iters - done))
        done += len(h)
        hist.append(h)
        cl, cd, _ = solver.forces(want_cp=False)
        forces.append((done, cl, cd))
    return np.concatenate(hist), forces


def run_residuals_only(args):
    """Evaluate the residual of the configured form args.residuals_only times
    from the timed start state (a small, fixed program to profile)."""
    import torch

    from paper_2403_13287_gb300 import lskum
    from paper_2403_13287_gb300.cloudgen import CLOUDS, naca0012_cloud, smooth_state
    torch.cuda.set_device(0)
    W, L = CLOUDS[args.workload]
    cloud = naca0012_cloud(W, L, shuffle=bool(args.shuffle))
    s = lskum.Solver(cloud, order=args.order, inner_iters=args.inner, time_scheme=1 if args.scheme == "rk4" else 0,
                     cfl=args.cfl, mach=args.mach, aoa_deg=args.aoa, reorder=args.reorder, limiter_K=args.limiter,
                     precision=1 if args.precision == "mixed" else 0)
    if args.precision == "mixed" and args.tuning != "auto":
        fv, qv = (int(v) for v in args.tuning.split(","))
        s.set_tuning(fv, qv)
    U = torch.from_numpy(smooth_state(cloud, args.mach, args.aoa, amp=0.05, seed=7)).cuda()
    for _ in range(args.residuals_only):
        s.residual(U)
    torch.cuda.synchronize()
    s.close()
    print(json.dumps({"residuals": args.residuals_only, "workload": args.workload, "points": int(cloud["n"]),
                      "precision": args.precision, "tuning": args.tuning}))
    return 0


def run_accuracy(args):
    """The mixed form's accuracy against the FP64 form on the 160k- and
    2.5M-point clouds (second order, 3 inner iterations, RK4, M 1.2, alpha 0,
    limiter K = 1). On the 160k cloud both forms run from the free stream to
    convergence. On the 2.5M cloud the mixed form runs from the free stream
    until its residue reaches its FP32 floor; then the FP64 form and the
    mixed form both continue from that state for the same number of
    iterations, and their forces are compared. Prints one JSON line."""
    import numpy as np
    import torch

    from paper_2403_13287_gb300 import lskum
    from paper_2403_13287_gb300.cloudgen import CLOUDS, naca0012_cloud
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    mach, aoa, lim = args.mach, args.aoa, args.limiter
    out = {"metric": "mixed-precision error against FP64 at convergence", "mach": mach, "aoa_deg": aoa,
           "limiter_K": lim, "order": args.order, "inner_iters": args.inner, "scheme": "rk4"}

    def solver(cloud, prec, cfl):
        s = lskum.Solver(cloud, order=args.order, inner_iters=args.inner, time_scheme=1, cfl=cfl, mach=mach,
                         aoa_deg=aoa, reorder=1, limiter_K=lim, precision=prec, stream=stream)
        if prec == 1:
            s.autotune(reps=3)
        return s

    def record(h, f, cp, t):
        return {"iterations": int(len(h)), "seconds": t, "residue_max": float(h.max()),
                "residue_last": float(h[-1]), "residue_drop": float(h[-1] / h.max()),
                "cl": f[-1][1], "cd": f[-1][2],
                "force_change_last_chunk": [abs(f[-1][1] - f[-2][1]), abs(f[-1][2] - f[-2][2])] if len(f) > 1
                else None, "forces": f[::max(1, len(f) // 12)] + f[-1:], "cp": cp}

    def errors(r64, rm):
        small_cl = aoa == 0.0
        return {"cl_rel_err": rel(rm["cl"], r64["cl"], r64["cd"] if small_cl else None),
                "cl_err_scale": "|Cd| (Cl ~ 0)" if small_cl else "|Cl|",
                "cd_rel_err": rel(rm["cd"], r64["cd"]),
                "cp_max_abs_err": float(np.max(np.abs(np.array(rm["cp"]) - np.array(r64["cp"]))))}

    for name, iters, cfl in (("naca0012_160k", args.acc_iters_160k, args.acc_cfl_160k),
                             ("naca0012_2p5m", args.acc_iters_2p5m, args.acc_cfl_2p5m)):
        if iters <= 0:
            continue
        W, L = CLOUDS[name]
        cloud = naca0012_cloud(W, L)
        res = {"points": int(cloud["n"]), "cfl": cfl}
        try:
            t0 = time.time()
            sm = solver(cloud, 1, cfl)
            hm, fm = converge(sm, iters, args.acc_chunk)
            cl, cd, cp = sm.forces()
            res["mixed"] = record(hm, fm, cp.tolist(), time.time() - t0)
            Um = sm.get_state()
            sm.close()
            t0 = time.time()
            s64 = solver(cloud, 0, cfl)
            if name == "naca0012_2p5m":
                # too slow to converge in FP64 here: both forms continue from
                # the mixed form's state for the same iterations, so that
                # the drift still left in the forces is the same for both
                # and their difference is the precision's
                n1 = args.acc_iters_fp64_restart
                s64.set_state(Um)
                h64, f64 = converge(s64, n1, args.acc_chunk)
                cl, cd, cp = s64.forces()
                res["fp64"] = record(h64, f64, cp.tolist(), time.time() - t0)
                s64.close()
                t0 = time.time()
                sm = solver(cloud, 1, cfl)
                sm.set_state(Um)
                hm2, fm2 = converge(sm, n1, args.acc_chunk)
                cl, cd, cp = sm.forces()
                res["mixed_continued"] = record(hm2, fm2, cp.tolist(), time.time() - t0)
                sm.close()
                res["fp64_started_from"] = ("the mixed form's state after %d iterations; mixed_continued runs "
                                            "the mixed form on from the same state" % iters)
                res["error"] = errors(res["fp64"], res["mixed_continued"])
                res["error_against_the_mixed_start_state"] = errors(res["fp64"], res["mixed"])
                res["mixed_continued"].pop("cp")
            else:
                h64, f64 = converge(s64, iters, args.acc_chunk)
                cl, cd, cp = s64.forces()
                res["fp64"] = record(h64, f64, cp.tolist(), time.time() - t0)
                s64.close()
                res["error"] = errors(res["fp64"], res["mixed"])
            for k in ("mixed", "fp64"):
                res[k].pop("cp")
        except lskum.LskumError as e:
            res["failed"] = str(e)
        out[name] = res
        print(json.dumps({name: res}), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)
    return 0


def batch_workload(n_clouds, n_cond, seed=240313292):
    """Seeded uneven batch: cloud sizes log-uniform in [20k, 400k] points
    (W:L about 2.6, as the single-cloud workloads), each under n_cond free
    streams with M uniform in [0.5, 1.2] and alpha uniform in [-2, 4] deg."""
    import numpy as np

    from paper_2403_13287_gb300.cloudgen import naca0012_cloud
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(20000.0), np.log(400000.0), n_clouds))
    cases = []
    for k, target in enumerate(sizes):
        W = max(32, int(round(math.sqrt(2.6 * target) / 8.0)) * 8)
        L = max(8, int(round(target / W)))
        c = naca0012_cloud(W, L, seed=seed + k)
        for _ in range(n_cond):
            cases.append((c, float(rng.uniform(0.5, 1.2)), float(rng.uniform(-2.0, 4.0))))
    return cases


def measure_batched(args, dist, sampler):
    """The batched form: all cases in one context (mixed precision, one
    autotuning), against the same cases stepped one context after another
    with the same launch shapes. Both timed over args.steps iterations with
    CUDA events on the library stream."""
    import numpy as np
    import torch

    from paper_2403_13287_gb300 import lskum
    from paper_2403_13287_gb300.cloudgen import smooth_state

    cases = batch_workload(args.batch_clouds, args.batch_conditions)
    stream = torch.cuda.current_stream()
    scheme = 1 if args.scheme == "rk4" else 0
    kw = dict(order=args.order, inner_iters=args.inner, time_scheme=scheme, cfl=args.cfl,
              limiter_K=args.limiter, precision=1, reorder=args.reorder, stream=stream.cuda_stream)
    U0 = [smooth_state(c, m, a, amp=0.05, seed=100 + k) for k, (c, m, a) in enumerate(cases)]
    npts = int(sum(c["n"] for c, _, _ in cases))

    def timed(fn):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist)

    B = lskum.Solver.batch(cases, **kw)
    B.set_state(np.concatenate(U0, axis=1))
    if args.tuning == "auto":
        tuning = B.autotune(reps=5)
    else:
        fv, qv = (int(v) for v in args.tuning.split(","))
        B.set_tuning(fv, qv)
        tuning = {"flux_variant": fv, "qgrad_variant": qv, "fixed": True}
    B.step(args.warmup, history=False)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    l0 = B.launch_count()
    ms_b = timed(lambda: B.step(args.steps, history=False))
    launches = B.launch_count() - l0
    clocks = sampler.stop() if sampler else None
    # idle share of the graph-replayed iteration: its time minus the summed
    # CUDA-event durations of its flux and q-derivative kernels (timed in a
    # separate, directly launched run; the residue kernels count as idle)
    B.profile(True)
    B.step(args.steps, history=False)
    fms, fn = B.kernel_time(lskum.LSKUM_KERNEL_FLUX)
    qms, qn = B.kernel_time(lskum.LSKUM_KERNEL_QGRAD)
    B.profile(False)
    B.close()
    gaps = {"graph_ms_per_iteration": ms_b / args.steps,
            "kernel_ms_per_iteration": (fms + qms) / args.steps,
            "launches_per_iteration": (fn + qn) / args.steps,
            "idle_share": max(0.0, 1.0 - (fms + qms) / ms_b)}

    singles = []
    for k, (c, m, a) in enumerate(cases):
        s = lskum.Solver(c, mach=m, aoa_deg=a, **kw)
        s.set_tuning(tuning["flux_variant"], tuning["qgrad_variant"])
        s.set_state(U0[k])
        s.step(args.warmup, history=False)
        singles.append(s)
    ms_s = timed(lambda: [s.step(args.steps, history=False) for s in singles])
    for s in singles:
        s.close()
    world = dist.get_world_size() if dist else 1
    value_b = replicas_value(npts, args.steps, ms_b, world)
    value_s = replicas_value(npts, args.steps, ms_s, world)
    sizes = sorted({int(c["n"]) for c, _, _ in cases})
    return {"value": value_b, "unit": UNIT, "ms_per_step": ms_b / args.steps, "dtype": "f32/f64 mixed",
            "cases": len(cases), "points": npts, "cloud_sizes": [sizes[0], sizes[-1]],
            "clouds": args.batch_clouds, "conditions_per_cloud": args.batch_conditions,
            "gpu_launches": launches, "tuning": tuning, "clocks": clocks, "launch_gaps": gaps,
            "sequential": {"value": value_s, "ms_per_step": ms_s / args.steps,
                           "note": "one context per case, stepped one after another with the same "
                                   "launch shapes; small cases then run from L2"},
            "speedup_vs_sequential": value_b / value_s}


def measure_adjoint(args, dist, sampler):
    """The adjoint form on the 640k-point cloud at M 0.63, alpha 2 (second
    order, RK4, unlimited; FP64): one residual VJP, one iteration VJP and a
    checkpointed reverse sweep through 16 iterations, each against the
    forward work it differentiates, with the device memory they add."""
    import numpy as np
    import torch

    from paper_2403_13287_gb300 import lskum
    from paper_2403_13287_gb300.adjoint import unrolled_force_gradient
    from paper_2403_13287_gb300.cloudgen import CLOUDS, naca0012_cloud, smooth_state

    W, L = CLOUDS["naca0012_640k"]
    cloud = naca0012_cloud(W, L)
    n = cloud["n"]
    mach, aoa = 0.63, 2.0
    stream = torch.cuda.current_stream()
    s = lskum.Solver(cloud, order=2, inner_iters=args.inner, time_scheme=1, cfl=args.cfl, mach=mach,
                     aoa_deg=aoa, reorder=1, limiter_K=0.0, precision=0, stream=stream.cuda_stream)
    U = torch.from_numpy(smooth_state(cloud, mach, aoa, amp=0.05, seed=9)).cuda()
    s.set_state(U)
    Rb = torch.from_numpy(np.random.default_rng(5).standard_normal((4, n))).cuda()

    def timed(fn, reps):
        fn()                                     # warm-up (allocates the workspace on first use)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / reps, dist)

    free0 = torch.cuda.mem_get_info()[0]
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ms_res = timed(lambda: s.residual(U), 5)
    ms_res_vjp = timed(lambda: s.residual_vjp(Rb, U), 3)
    free1 = torch.cuda.mem_get_info()[0]
    # the FP32 product, on a mixed context of the same cloud
    sm = lskum.Solver(cloud, order=2, inner_iters=args.inner, time_scheme=1, cfl=args.cfl, mach=mach,
                      aoa_deg=aoa, reorder=1, limiter_K=0.0, precision=1, stream=stream.cuda_stream)
    ms_res_m = timed(lambda: sm.residual(U), 5)
    ms_res_vjp32 = timed(lambda: sm.residual_vjp(Rb, U, fp32=True), 3)
    sm.close()
    # the limited scheme (K = 1) at the supersonic condition: the residual VJP
    # through the limiter, on the same cloud
    sl = lskum.Solver(cloud, order=2, inner_iters=args.inner, time_scheme=1, cfl=args.cfl, mach=1.2,
                      aoa_deg=0.0, reorder=1, limiter_K=1.0, precision=0, stream=stream.cuda_stream)
    Ul = torch.from_numpy(smooth_state(cloud, 1.2, 0.0, amp=0.05, seed=9)).cuda()
    ms_res_l = timed(lambda: sl.residual(Ul), 5)
    ms_res_vjp_l = timed(lambda: sl.residual_vjp(Rb, Ul), 3)
    sl.close()
    ms_step = timed(lambda: s.step(1, history=False), 3)
    s.set_state(U)
    ms_step_vjp = timed(lambda: s.step_vjp(Rb, U), 3)
    free2 = torch.cuda.mem_get_info()[0]
    iters = 16
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    (cl, cd), (Ub, xb, yb), info = unrolled_force_gradient(s, U, iters)
    torch.cuda.synchronize()
    sweep_s = max_over_ranks(time.perf_counter() - t0, dist)
    clocks = sampler.stop() if sampler else None
    s.close()
    return {"workload": "naca0012_640k", "points": n, "mach": mach, "aoa_deg": aoa, "scheme": "rk4",
            "dtype": "f64", "residual_ms": ms_res, "residual_vjp_ms": ms_res_vjp,
            "residual_vjp_over_residual": ms_res_vjp / ms_res,
            "mixed_residual_ms": ms_res_m, "residual_vjp_fp32_ms": ms_res_vjp32,
            "fp32_vjp_speedup": ms_res_vjp / ms_res_vjp32,
            "limited_m12": {"residual_ms": ms_res_l, "residual_vjp_ms": ms_res_vjp_l,
                            "residual_vjp_over_residual": ms_res_vjp_l / ms_res_l,
                            "note": "limiter K = 1, M 1.2, alpha 0: the VJP through the limiter"},
            "iteration_ms": ms_step,
            "iteration_vjp_ms": ms_step_vjp, "iteration_vjp_over_iteration": ms_step_vjp / ms_step,
            "residual_vjp_workspace_bytes": free0 - free1, "iteration_vjp_workspace_bytes": free1 - free2,
            "unrolled": {"iterations": iters, "seconds": sweep_s, "cl": cl, "checkpoint_every": info["checkpoint_every"],
                         "recomputed_iterations": info["recomputed_iterations"],
                         "state_bytes_peak": info["state_bytes_peak"],
                         "state_bytes_unrolled": info["state_bytes_unrolled"]},
            "clocks": clocks}


def run_ours(args, rank, world, local):
    import torch

    from paper_2403_13287_gb300.cloudgen import CLOUDS, naca0012_cloud

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    W, L = CLOUDS[args.workload]
    cloud = naca0012_cloud(W, L, shuffle=bool(args.shuffle))
    n = cloud["n"]
    dbar = cloud["nbr_offsets"][-1] / n
    primary = args.precision
    other = "mixed" if primary == "fp64" else "fp64"
    peaks, peak_src = measured_peaks()
    from paper_2403_13287_gb300 import lskum as _lskum
    probes = {"fp64_fma_gflops": _lskum.probe_peak(_lskum.PROBE_FP64_FMA),
              "fp32_fma_gflops": _lskum.probe_peak(_lskum.PROBE_FP32_FMA),
              "fp32x2_fma_gflops": _lskum.probe_peak(_lskum.PROBE_FP32X2_FMA)}

    rp = measure_form(args, cloud, primary, dist, ClockSampler(local) if rank == 0 else None)
    tuning = rp.get("tuning")
    e2e_value = world * measure_e2e(rp["solver"], n, max(1, args.steps), dist)
    rp["solver"].close()
    forms = {primary: form_summary(args, rp, n, dbar, world, primary, peaks, peak_src, probes)}
    if not args.single_form:
        ro = measure_form(args, cloud, other, dist, ClockSampler(local) if rank == 0 else None)
        ro["solver"].close()
        forms[other] = form_summary(args, ro, n, dbar, world, other, peaks, peak_src, probes)
        forms[other]["clocks"] = ro["clocks"]
        if ro.get("tuning"):
            forms[other]["tuning"] = ro["tuning"]
        forms["mixed_speedup_vs_fp64"] = forms["mixed"]["value"] / forms["fp64"]["value"]
        if not args.no_error:
            forms["mixed"]["error"] = measure_mixed_error(
                args, cloud, forms["mixed"].get("tuning") or tuning, torch.cuda.current_stream().cuda_stream)
    if not args.no_batch and not args.single_form:
        forms["batched"] = measure_batched(args, dist, ClockSampler(local) if rank == 0 else None)
        forms["batched_speedup_vs_fp64"] = forms["batched"]["value"] / forms["fp64"]["value"]
        forms["batched"]["error"] = ("the mixed form's (forms.mixed.error): every case of a batch gives, bit for "
                                     "bit, the states of a mixed context of its own (tests/test_gpu_batch.py)")
    if not args.no_adjoint and not args.single_form:
        forms["adjoint"] = measure_adjoint(args, dist, ClockSampler(local) if rank == 0 else None)
    if not args.no_extra and not args.single_form:
        import copy

        def variant(precision, cl, **over):
            a = copy.copy(args)
            for k, v in over.items():
                setattr(a, k, v)
            r = measure_form(a, cl, precision, dist, ClockSampler(local) if rank == 0 else None)
            r["solver"].close()
            nn = cl["n"]
            out = form_summary(a, r, nn, cl["nbr_offsets"][-1] / nn, world, precision, peaks, peak_src, probes)
            out["clocks"] = r["clocks"]
            if r.get("tuning"):
                out["tuning"] = r["tuning"]
            out["config"] = {k: getattr(a, k) for k in ("scheme", "mach", "aoa", "limiter", "reorder")}
            out["config"]["boundary"] = "kinetic" if getattr(a, "boundary", 0) else "plain"
            out["config"]["points"] = nn
            return out

        # the paper's own benchmark condition: 2nd order, 3 inner iterations,
        # forward Euler, M 0.63, alpha 2, no limiter (its A100 figures are FP64)
        fe = {p_: variant(p_, cloud, scheme="euler", mach=0.63, aoa=2.0, limiter=0.0) for p_ in ("fp64", "mixed")}
        fe["paper_a100_cuda_c_fp64"] = {"2M": 1.52e8, "4M": 1.81e8, "unit": UNIT,
                                        "note": "context: A100, FP64, the paper's clouds; not this GPU or cloud"}
        forms["forward_euler_m063"] = fe
        # ablation of the numbering: the shuffled input order kept, and reverse Cuthill-McKee
        forms["mixed_input_order"] = variant("mixed", cloud, reorder=0)
        forms["mixed_input_order"]["speedup_of_morton"] = forms["mixed"]["value"] / forms["mixed_input_order"]["value"]
        forms["mixed_rcm"] = variant("mixed", cloud, reorder=2)
        forms["mixed_rcm"]["speedup_of_morton"] = forms["mixed"]["value"] / forms["mixed_rcm"]["value"]
        # the kinetic boundary mode (mirror images at the wall and far-field points)
        kin = {p_: variant(p_, cloud, boundary=1) for p_ in ("fp64", "mixed")}
        for p_ in ("fp64", "mixed"):
            kin[p_]["relative_to_plain"] = kin[p_]["value"] / forms[p_]["value"]
        forms["kinetic_boundary"] = kin
        # throughput at 10M points
        W10, L10 = CLOUDS["naca0012_10m"]
        c10 = naca0012_cloud(W10, L10, shuffle=bool(args.shuffle))
        forms["mixed_10m"] = variant("mixed", c10)
        del c10
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    main = forms[primary]
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": main["dtype"], "data": "synthetic",
        "config": {"workload": args.workload, "points": n, "mean_degree": round(float(dbar), 3),
                   "order": args.order, "inner_iters": args.inner, "scheme": args.scheme,
                   "mach": args.mach, "aoa_deg": args.aoa, "cfl": args.cfl, "limiter_K": args.limiter,
                   "precision": primary, "reorder": "morton" if args.reorder else "none",
                   "input_order": "shuffled" if args.shuffle else "structured",
                   "l2": "inputs larger than L2 (working set ~%.1f GB)" % (
                       (n * 380 + cloud["nbr_offsets"][-1] * 37) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "edge_iterations_per_s": main["edge_iterations_per_s"],
        "roofline": main["roofline"],
        "kernels": main["kernels"],
        "gpu_launches": main["gpu_launches"],
        "measured_fma_peaks_gflops": probes,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n * 8,
                "d2h_bytes_per_step": 4 * n * 8 + 8},
        "clocks": rp["clocks"],
        "forms": {k: v for k, v in forms.items() if k != primary},
    }
    if tuning:
        line["tuning"] = tuning
    if not args.no_cpu_baseline and world == 1:
        import oracle
        m = oracle.split_stencils(cloud)
        line["cpu_baseline"] = cpu_baseline_sample(cloud, m, args)
    line["summary"] = summary_of(line, forms)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.gpus != world and world > 1:
        print("warning: --gpus %d but WORLD_SIZE %d" % (args.gpus, world), file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.accuracy:
        return run_accuracy(args)
    if args.residuals_only:
        return run_residuals_only(args)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
