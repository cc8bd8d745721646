#!/usr/bin/env python3
"""Throughput of the FGA hot path on one GB300: Gaussian.gridpoint evaluations per second.

One step = the whole path on one batch of synthetic input: decompose (FBI,
branch split, thresholding), propagate (RK4 rays, dynamic rays, amplitude,
action) and reconstruct (binning + gather on the grid). The workload is the
layered model (737 x 241 at 12.5 m, 12 dipping layers, 3 faults, smoothed),
one 15 Hz Ricker-ring source at 10 m depth, eps from 15 Hz, T = 2 s, dt = 1 ms,
tau = 1e-3, kappa = 6.

A Gaussian.gridpoint evaluation is one (Gaussian, grid point) pair inside the
Gaussian's kappa*sqrt(eps) square window, counted over both branches of the
method (the GPU evaluates the + branch and obtains the - branch as its complex
conjugate).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica of the workload (the
shots are independent problems, no collective on the data path); value is the
evaluations of all ranks divided by the slowest rank's time. --impl reference
times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (rank 0 only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1304_3542_gb300.workloads import window_evals  # noqa: E402

METRIC = "FGA Gaussian·gridpoint evals/s and rel-L2 err; mixed-prec vs FP64, 1 GB300"
UNIT = "evals/s"
L2_FLUSH_BYTES = 256 << 20
# FP64 operations of one RK4 ray step in 2D, counted from the source of the ray
# kernel (add/sub/mul/rsqrt/reciprocal = 1, fma = 2; conversions, compares and the
# Newton steps that refine the hardware's rsqrt and reciprocal not counted): 4
# right-hand sides of 280 (medium from the per-cell polynomial table 86: cell offsets 8,
# four rows in z by Horner with derivatives 48, combination in x 30; |P|, n, dQ/dt,
# dP/dt and -|P| K 18; dynamic rays 96; Z, dZ/dt, tr(adj Z dZ/dt) and det Z 60; da/dt
# 20) plus 308 for the stage combinations of the 22 integrated state values (7 fma
# each; the action S has a right-hand side that vanishes identically and is carried, not
# integrated).
FLOPS_PER_RAY_STEP_2D = 1428
# FP64 peak from the unit counts and clocks: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def workload():
    from paper_1304_3542_gb300 import workloads as WL

    return WL.layered_single()


def workload_name(prob):
    sh = prob.shots[0]
    return ("layered model %dx%d at %.1f m, 1 shot %g Hz Ricker ring at (%.2f, %.2f) km, "
            "T=%g s, dt=%g s" % (prob.n[0], prob.n[1], prob.h[0] * 1000, sh.freq, sh.source[0],
                                  sh.source[1], prob.T, prob.dt))


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch of the ray kernel from the committed ncu summary, if it was
    taken on the kernel source as it is now (else None)."""
    path = os.path.join(ROOT, "profiles", "k_rays_layered_single.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        cur = source_hash(rec["sources"])
        if rec.get("source_hash") != cur:
            return None
        return rec.get("dram_bytes_per_launch")
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1304_3542_gb300 import fga as F

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = workload()
    stream = torch.cuda.current_stream(dev)
    precision = F.FGA_MIXED_TF32X3 if args.precision == "mixed" else F.FGA_FP64
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=precision)
    u0, u1 = F.stacked_initial_data(prob)
    d_u0 = torch.from_numpy(u0).to(dev)
    d_u1 = torch.from_numpy(u1).to(dev)
    d_out = torch.zeros((1,) + prob.n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(a, b, out):
        plan.decompose(a, b)
        plan.propagate()
        plan.reconstruct(out)

    # first pass: the autotuner picks the ray launch shape and the gather's segment
    # length on this workload; then the Gaussian count and evaluation count
    plan.decompose(d_u0, d_u1)
    tuning = plan.autotune(d_out)
    step(d_u0, d_u1, d_out)
    plan.sync()
    G = plan.count(0)
    st = plan.state(0)
    evals_plus = window_evals(prob, st["Q"], prob.shots[0].eps)
    evals = 2.0 * evals_plus
    for _ in range(args.warmup):
        step(d_u0, d_u1, d_out)
    plan.sync()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    _, launches0 = plan.stage_times()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ray_ms, recon_ms, fbi_ms, ray_steps = [], [], [], []
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))  # L2 flush between timed steps (outside the events)
            starts[i].record(stream)
            step(d_u0, d_u1, d_out)
            ends[i].record(stream)
            stt, _ = plan.stage_times()
            ray_steps.append(plan.ray_steps())
            ray_ms.append(stt["rays"])
            recon_ms.append(stt["reconstruct"] + stt["binning"])
            fbi_ms.append(stt["fbi"])
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    _, launches1 = plan.stage_times()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * evals * args.steps / total_s
    ms_per_step = total_s * 1e3 / args.steps

    # end to end through the C ABI with host buffers (pinned), copies inside the timing
    h_u0 = torch.from_numpy(u0).pin_memory()
    h_u1 = torch.from_numpy(u1).pin_memory()
    h_out = torch.empty((1,) + prob.n, dtype=torch.float64).pin_memory()
    e2e_times = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        step(h_u0, h_u1, h_out)  # reconstruct into host memory waits for the copy
        e2e_times.append(time.perf_counter() - t1)
    e2e_s = sum(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * evals * args.steps / e2e_s
    npts = prob.npoints

    rel_l2 = None
    fp64_value = None
    if precision != F.FGA_FP64:
        # the FP64 path on the same input: the reference for the mixed path's error
        ref = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=F.FGA_FP64)
        d_ref = torch.zeros_like(d_out)
        ref.decompose(d_u0, d_u1)
        ref.autotune(d_ref)
        ref.sync()
        rel_l2 = float((d_out - d_ref).norm() / d_ref.norm())
        t64 = []
        for i in range(max(1, args.steps)):
            flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ref.decompose(d_u0, d_u1)
            ref.propagate()
            ref.reconstruct(d_ref)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1) / 1e3)
        fp64_value = evals / statistics.mean(t64)
        ref.close()
    # the FMA pipes measured on this GPU in this run (roofline denominators' check)
    fp64_meas, _ = F.fma_peak(64, 4096)
    fp32_meas, _ = F.fma_peak(32, 65536)
    ray_s = statistics.mean(ray_ms) / 1e3
    steps_done = statistics.mean(ray_steps)
    ray_flops = FLOPS_PER_RAY_STEP_2D * steps_done
    achieved = ray_flops / ray_s / 1e12
    clocks = clk.summary()
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if precision == F.FGA_FP64 else "f64+tf32",
        "data": "synthetic (seeded layered model and Ricker ring; no dataset)",
        "rel_l2_vs_fp64": rel_l2,
        "config": {
            "workload": workload_name(prob),
            "grid": list(prob.n),
            "eps_km": prob.shots[0].eps,
            "q_stride": list(prob.shots[0].q_stride),
            "box": list(prob.shots[0].box),
            "tau": prob.tau,
            "kappa": prob.kappa,
            "gaussians_plus_branch": G,
            "ray_steps_integrated": steps_done,
            "ray_steps_all_to_T": G * prob.nsteps,
            "evals_per_step_both_branches": evals,
            "precision": ("fp64" if precision == F.FGA_FP64 else
                          "mixed: FBI stage 2 and the reconstruction on tensor cores "
                          "(TF32 head/tail operands, 3 products, FP32 accumulate; FP64 phase "
                          "anchors and segment sums); FBI stage 1 in FP32 on the CUDA cores, "
                          "psi stored as FP32 pairs; selection and rays FP64"),
            "fp64_path_value": fp64_value,
            "tuning": {"ray_blocks_per_sm": tuning[0], "gather_segment": tuning[1],
                       "ray_register_variant": tuning[2],
                       "by": "fga_autotune on this workload before the warm-up"},
            "stage_ms_mean": {"fbi": statistics.mean(fbi_ms), "rays": statistics.mean(ray_ms),
                              "binning+reconstruct": statistics.mean(recon_ms)},
            "l2": "256 MiB buffer written between timed steps",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "wall_s_timed_region": wall,
        },
        "roofline": {
            "kernel": "k_rays<2> (RK4 rays, dynamic rays, amplitude, action)",
            "bound": "alu",
            "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": ncu_traffic(),
            "flops_per_launch": ray_flops,
            "peak_source": ("FP64 from unit counts and clock (152 SM x 2 DFMA/clk x 2.07 GHz); "
                            "the same figure measured by fga_fma_peak, 1.2553 and 1.2572 "
                            "TFLOP/s (profiles/fma_peak_microbenchmark.md), and again in "
                            "this run (peak_measured)"),
            "peak_measured": {"fp64_tflops": fp64_meas, "fp32_tflops": fp32_meas,
                              "frac_of_measured_fp64": achieved / fp64_meas,
                              "by": "fga_fma_peak (csrc/fga_peaks.cu): 8 FMA chains per "
                                    "thread, 8 x 256 threads per SM, CUDA events, this run"},
        },
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * npts,
                "d2h_bytes_per_step": 8 * npts},
        "gpu_launches": int(launches1 - launches0),
        "clocks": clocks,
    }
    plan.close()
    return line, prob, evals


def oracle_sample(prob, n_sample, nthreads):
    """One bounded oracle pass: the full decomposition, then n_sample Gaussians (half
    of each branch) propagated to T and summed on every grid point. Returns
    (estimated seconds for the whole workload, description, evals of the workload)."""
    import oracle as O

    sh = prob.shots[0]
    g = O.Grid(prob.n, prob.h, prob.origin, prob.periodic)
    nz = (sh.u0 != 0) | (sh.u1 != 0)
    nq = O.q_counts(g, sh.q_stride)
    keep = []
    for k in range(prob.dim):
        other = tuple(a for a in range(prob.dim) if a != k)
        idx = np.flatnonzero(np.any(nz, axis=other))
        m = np.arange(nq[k]) * sh.q_stride[k]
        keep.append((m - sh.box[k] // 2 <= idx.max()) & (m + sh.box[k] // 2 - 1 >= idx.min()))
    mesh = np.meshgrid(*keep, indexing="ij")
    rows = np.flatnonzero(np.logical_and.reduce([x.ravel() for x in mesh]))
    t0 = time.perf_counter()
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau,
                      q_subset=rows)
    t_dec = time.perf_counter() - t0
    gs = dec["gauss"]
    G2 = gs["sigma"].size
    rng = np.random.default_rng(1304)
    pick = np.concatenate([rng.choice(np.flatnonzero(gs["sigma"] == s), n_sample // 2,
                                      replace=False) for s in (1, -1)])
    t0 = time.perf_counter()
    st = O.propagate(g, prob.velocity, prob.nsteps, prob.dt, gs["sigma"][pick], gs["q"][pick],
                     gs["p"][pick], nthreads)
    t_prop = time.perf_counter() - t0
    W = O.quadrature_weight(g, sh.eps, sh.q_stride, sh.box)
    t0 = time.perf_counter()
    O.reconstruct(g, sh.eps, prob.kappa, W, st["Q"], st["P"], st["a"], gs["psi"][pick], st["S"],
                  prob.grid_points(), nthreads)
    t_rec = time.perf_counter() - t0
    scale = G2 / pick.size
    est = t_dec + scale * (t_prop + t_rec)
    evals_sample = window_evals(prob, st["Q"], sh.eps)
    evals = evals_sample * scale
    desc = ("full decomposition (%.1f s) + %d of %d Gaussians propagated %d steps (%.1f s) and "
            "summed on all %d grid points (%.1f s), time scaled by %.0fx"
            % (t_dec, pick.size, G2, prob.nsteps, t_prop, prob.npoints, t_rec, scale))
    return est, desc, evals, t_dec + t_prop + t_rec


def measure_batch(prob, dev, reps):
    """The batched forms on the shots of prob: mixed precision with all shots in one plan
    and decompose + propagate + reconstruct replayed as one CUDA graph (fga_run_pipeline),
    against FP64 with all shots in one plan (eager) and FP64 one plan per shot. One
    untimed pass of each form (it captures the graph), then reps timed passes; CUDA
    events on the plans' stream, a 256 MiB L2 flush between passes."""
    import dataclasses

    import torch

    from paper_1304_3542_gb300 import fga as F

    stream = torch.cuda.Stream(dev)
    u0, u1 = F.stacked_initial_data(prob)
    d_u0, d_u1 = torch.from_numpy(u0).to(dev), torch.from_numpy(u1).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        out = []
        for i in range(reps):
            flush.fill_(float(i))
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1) / 1e3)
        return statistics.mean(out)

    ns = len(prob.shots)
    with torch.cuda.stream(stream):
        mixed = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=F.FGA_MIXED_TF32X3)
        d_mx = torch.zeros((ns,) + prob.n, dtype=torch.float64, device=dev)
        mixed.decompose(d_u0, d_u1)
        tuning = mixed.autotune(d_mx)
        mixed.run_pipeline(d_u0, d_u1, d_mx)  # eager sizing pass and capture
        mixed.sync()
        counts = [mixed.count(s) for s in range(ns)]
        evals = 0.0
        for s in range(ns):
            evals += 2.0 * window_evals(prob, mixed.state(s)["Q"], prob.shots[s].eps)
        _, l0 = mixed.stage_times()
        t_mixed = timed(lambda: mixed.run_pipeline(d_u0, d_u1, d_mx))
        mixed.sync()
        _, l1 = mixed.stage_times()
        mixed.close()  # free its buffers before the FP64 forms
        b64 = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=F.FGA_FP64)
        d_64 = torch.zeros_like(d_mx)
        b64.decompose(d_u0, d_u1)
        b64.autotune(d_64)

        def b64_step():
            b64.decompose(d_u0, d_u1)
            b64.propagate()
            b64.reconstruct(d_64)

        t_b64 = timed(b64_step)
        rel = float((d_mx - d_64).norm() / d_64.norm())
        b64.close()
        singles = []
        for s in range(ns):
            one = dataclasses.replace(prob, shots=[prob.shots[s]])
            singles.append(F.plan_from_problem(one, stream=stream.cuda_stream,
                                               precision=F.FGA_FP64))

        def per_shot_step():
            for s, pl in enumerate(singles):
                pl.decompose(d_u0[s:s + 1], d_u1[s:s + 1])
                pl.propagate()
                pl.reconstruct(d_64[s:s + 1])

        per_shot_step()
        t_single = timed(per_shot_step)
        for pl in singles:
            pl.close()
    return {
        "evals": evals, "t_mixed": t_mixed, "rel_l2_mixed_vs_fp64": rel,
        "gaussians_per_shot": {"min": min(counts), "median": statistics.median(counts),
                               "max": max(counts)},
        "tuning": {"ray_blocks_per_sm": tuning[0], "gather_segment": tuning[1],
                   "ray_register_variant": tuning[2]},
        "kernel_launches_per_replay": int((l1 - l0) // max(reps, 1)),
        "seconds_per_pass": {"mixed_batched_pipeline_graph": t_mixed, "fp64_batched": t_b64,
                             "fp64_one_plan_per_shot": t_single},
        "speedup_batching_fp64": t_single / t_b64,
        "speedup_precision_batched": t_b64 / t_mixed,
        "speedup_total_vs_fp64_per_shot": t_single / t_mixed,
    }


def run_batch(args, rank, world, local_rank):
    """The batched-shots workload (64 shots on the layered model, per-shot frequency and
    eps): this rank's shots (contiguous block, no collective) in the three forms of
    measure_batch; value is the mixed pipeline-graph form's evaluations per second."""
    import dataclasses

    import torch

    from paper_1304_3542_gb300 import workloads as WL
    from paper_1304_3542_gb300.shards import max_over_ranks, shard_shots

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    full = WL.layered_batch()
    mine = shard_shots(len(full.shots), rank, world)
    prob = dataclasses.replace(full, shots=[full.shots[i] for i in mine])
    m = measure_batch(prob, dev, args.steps)
    t_mixed_all = max_over_ranks(m["t_mixed"])
    evals_all = m["evals"]
    if world > 1:
        t = torch.tensor([m["evals"]], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t)
        evals_all = float(t.item())
    cfg = {
        "workload": "layered model 737x241 at 12.5 m, 64 shots (x ~ U(1.0, 8.2) km, depth ~ "
                    "U(0.01, 0.5) km, f ~ U(8, 25) Hz, per-shot eps), T=2 s, dt=1 ms",
        "shots_this_rank": len(mine),
        "form": "mixed precision, all shots of the rank in one plan, decompose + propagate + "
                "reconstruct replayed as one CUDA graph with the counts on the device",
        "l2": "256 MiB buffer written between timed passes",
        "parallelism": "shot-parallel, %d rank(s), no collective" % world,
    }
    cfg.update({k: v for k, v in m.items() if k not in ("evals", "t_mixed", "rel_l2_mixed_vs_fp64")})
    return {
        "metric": METRIC,
        "value": evals_all / t_mixed_all,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": 1,
        "ms_per_step": t_mixed_all * 1e3,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f64+tf32",
        "data": "synthetic (seeded layered model, 64 Ricker-ring shots; no dataset)",
        "rel_l2_vs_fp64": m["rel_l2_mixed_vs_fp64"],
        "config": cfg,
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    prob = workload()
    cores = os.cpu_count() or 1
    vals, ests = [], []
    for i in range(args.warmup + args.steps):
        # the same sample (size and seed) as the cpu_baseline leg of the GPU line
        est, desc, evals, spent = oracle_sample(prob, args.cpu_sample, cores)
        if i >= args.warmup:
            vals.append(evals / est)
            ests.append(est)
    value = statistics.mean(vals)
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 * statistics.mean(ests),
        "ms_per_step_kind": "a whole step projected from the timed sample (see cpu_baseline.sample)",
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded layered model and Ricker ring; no dataset)",
        "config": {"workload": workload_name(prob), "grid": list(prob.n),
                   "eps_km": prob.shots[0].eps, "q_stride": list(prob.shots[0].q_stride),
                   "box": list(prob.shots[0].box), "tau": prob.tau, "kappa": prob.kappa,
                   "precision": "fp64",
                   "parallelism": "CPU oracle, OpenMP over Gaussians / grid points"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=512)
    ap.add_argument("--batch-shots", type=int, default=8,
                    help="shots of the batched workload timed in the three batched forms "
                         "for the line's batch sub-record (0: none; N = 1 only)")
    ap.add_argument("--workload", choices=["layered_single", "layered_batch"],
                    default="layered_single",
                    help="layered_batch: the 64-shot batched form against FP64 batched and "
                         "FP64 one plan per shot (one timed pass each by default)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed",
                    help="mixed: tensor-core reconstruction (its rel-L2 against the FP64 "
                         "path is measured in the same run); fp64: every step in FP64")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if args.impl == "ours":
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return
    if args.workload == "layered_batch":
        line = run_batch(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
            dist.destroy_process_group()
        return
    line, prob, evals = run_ours(args, rank, world, local_rank)
    if world == 1 and args.batch_shots > 0:
        import torch

        from paper_1304_3542_gb300 import workloads as WL

        full = WL.layered_batch()
        sub = full.with_(shots=full.shots[:args.batch_shots])
        m = measure_batch(sub, torch.device("cuda", local_rank), 1)
        m["value"] = m.pop("evals") / m["t_mixed"]
        m["unit"] = UNIT
        m["shots"] = "the first %d of the 64 shots of the batched workload (layered model, "\
                     "x ~ U(1.0, 8.2) km, depth ~ U(0.01, 0.5) km, f ~ U(8, 25) Hz, T = 2 s); "\
                     "one timed pass per form" % args.batch_shots
        line["batch"] = m
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            est, desc, ev_o, spent = oracle_sample(prob, args.cpu_sample, cores)
            line["cpu_baseline"] = {"value": ev_o / est, "unit": UNIT, "cores": cores,
                                    "kind": "oracle", "sample": desc}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
