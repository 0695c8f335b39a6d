#!/usr/bin/env python
"""Fisher-BT benchmark on GB300: FP64-accurate against mixed precision at matched theta_hat.

A step is one Fisher-BT iteration of Algorithm 1 (Sec. 2.1) over the whole hot path: the
backtracking line search (Algorithm 2 per candidate: covariance generation, tiled Cholesky,
log-determinant, triangular solve) followed by the Fisher scoring iteration at the accepted point
(Algorithm 3: Sigma_alpha / Sigma_nu, back-solve, quadratic forms, the two-sided transforms with
trace / Frobenius epilogues, assembly) and the 3x3 solve for the next direction.  Every timed step
starts from the same state (theta^(0) of the workload, its l, score, Fisher and direction), so
every step does the same work.

The line's value is the FP64-accurate path's iterations/s (tile products from exact BF16 digit
products on the tensor cores); beside it, in the same line, the mixed path's iterations/s, both
paths' Fisher-BT estimates from theta^(0) (Algorithm 1 to the paper's stopping rule; the mixed run
switches to FP64-accurate products once its steps are small) and the Cholesky rate.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload NAME]

Default workload: n = 65,536 uniform locations on [0,1]^2 (seed 2), field z ~ N(0, Sigma) at
theta_true = (1, 0.05, 0.8) with 1e-8 jitter, start theta^(0) = (0.7, 0.035, 0.64).  N > 1 runs N
independent replicas (one per GPU, launched by torchrun); the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import copy
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the batched modes drive up to 64 streams at once; the runtime maps streams onto this many
# hardware queues (default 8) when the CUDA context is created
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from paper_2601_11437_gb300 import inputs  # noqa: E402

FIELDS = os.path.join(ROOT, "tests", "golden", "fields")
METRIC = "Fisher-BT iters/s and Cholesky TFLOP/s (% peak): FP64 vs mixed at matched theta_hat"
PRECISIONS = {"fp64": 0, "fp64_emulated": 1, "mixed": 2}
# tensor-core work of one emulated FP64 tile product: 28 BF16 digit products of the same shape
OZAKI_PRODUCTS = 28
# DRAM bytes per 128 x 64 task of the emulated-FP64 tile update, from the ncu capture of one
# launch of the two-sided transform's trailing update at n = 4096 (156.671 MB read + 72.038 MB
# written over the launch's 1984 tasks); the C tiles, which dominate it, grow in proportion to
# the tasks
OZAKI_DRAM_BYTES_PER_TASK = (156.67072e6 + 72.0384e6) / 1984
OZAKI_TASK_FLOPS = 2.0 * 128 * 64 * 128
# FP64 peak for the roofline: the DFMA pipe, 2 FP64 FMA per clock per SM (measured on GB300:
# 1.19 TFLOP/s sustained at ~1.99 GHz), 152 SMs, 2 flop per FMA, 2.07 GHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# subsample sizes of the oracle's timing (CPU baseline and reference arm): its time per iteration
# is fitted as t(n) = a n^2 + b n^3 (generation O(n^2), dense algebra O(n^3)) and taken to n
ORACLE_SIZES = (1024, 2048, 4096)


def load_field(name: str):
    w = inputs.WORKLOADS[name]
    locs = w.locations()
    path = os.path.join(FIELDS, f"{name}_z.npy")
    meta = json.load(open(os.path.join(FIELDS, f"{name}_z.json")))
    sha = hashlib.sha256(np.ascontiguousarray(locs, dtype="<f8").tobytes()).hexdigest()
    if sha != meta["locations_sha256"]:
        raise RuntimeError(f"stored field {path} does not belong to these locations")
    return w, locs, np.load(path)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world, device):
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.barrier(device_ids=[device])
        torch.cuda.synchronize()


def max_over_ranks(world, value, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=f"cuda:{device}")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_step_seconds(locs, z, w, n_sub, seed_sub):
    """One oracle Fisher-BT iteration (line search + Algorithm 3) on a seeded subsample; the
    field restricted to a subset of locations is a draw of the model on that subset."""
    from oracle import fisher_bt, likelihood
    idx = inputs.subsample(w, n_sub, seed_sub)
    ev = likelihood.DenseEvaluator(locs[idx], z[idx])
    st0 = fisher_bt.start(ev, theta0=w.theta0)
    st = copy.deepcopy(st0)
    t0 = time.perf_counter()
    fisher_bt.step(ev, st)
    return time.perf_counter() - t0, st.n_ll - st0.n_ll


def oracle_extrapolation(times: dict, n: int):
    """Least-squares fit t(m) = a m^2 + b m^3 (a, b >= 0) to the oracle's mean iteration time at
    each measured subsample size m, evaluated at n."""
    ms = np.array(sorted(times), dtype=float)
    ts = np.array([np.mean(times[m]) for m in sorted(times)])
    A = np.stack([ms ** 2, ms ** 3], axis=1)
    coef, *_ = np.linalg.lstsq(A / ts[:, None], np.ones_like(ts), rcond=None)   # relative residuals
    a, b = max(coef[0], 0.0), max(coef[1], 0.0)
    if a == 0.0 and b == 0.0:
        b = float(ts[-1] / ms[-1] ** 3)
    return a * n ** 2 + b * n ** 3, a, b


def cores_used():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baseline(locs, z, w, sizes=ORACLE_SIZES):
    """The oracle's Fisher-BT iteration at each subsample size once, extrapolated to the
    workload's n (the reference arm uses the same sizes and rule)."""
    times = {m: [cpu_oracle_step_seconds(locs, z, w, m, 3)[0]] for m in sizes}
    t_full, a, b = oracle_extrapolation(times, w.n)
    meas = ", ".join(f"n={m}: {times[m][0]:.1f} s" for m in sizes)
    return {"value": 1.0 / t_full, "unit": "iters/s", "cores": cores_used(), "kind": "oracle",
            "sample": (f"one oracle Fisher-BT iteration (numpy FP64; BLAS threads for the matrix products) "
                       f"on seeded subsamples of the workload ({meas}), fitted by t = a n^2 + b n^3 "
                       f"(a = {a:.3e}, b = {b:.3e}) and evaluated at n = {w.n}: {t_full:.0f} s per iteration")}


def run_reference(args):
    """The oracle as the reference arm: each step one oracle Fisher-BT iteration on a seeded
    subsample, the sizes of ORACLE_SIZES in turn; the iterations/s at the workload's n come from
    the fitted time per iteration, the same rule as the native arm's cpu_baseline."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, locs, z = load_field(args.workload)
    sizes = args.reference_sizes
    for i in range(args.warmup):
        cpu_oracle_step_seconds(locs, z, w, sizes[0], 3)
    times = {m: [] for m in sizes}
    t0 = time.perf_counter()
    for i in range(args.steps):
        m = sizes[i % len(sizes)]
        times[m].append(cpu_oracle_step_seconds(locs, z, w, m, 3)[0])
    wall = time.perf_counter() - t0
    times = {m: v for m, v in times.items() if v}
    if len(times) >= 2:
        t_full, a, b = oracle_extrapolation(times, w.n)
        rule = f"fitted by t = a n^2 + b n^3 (a = {a:.3e}, b = {b:.3e})"
    else:
        (m, v), = times.items()
        t_full = float(np.mean(v)) * (w.n / m) ** 3
        rule = f"scaled by (n/{m})^3"
    value = 1.0 / t_full
    meas = ", ".join(f"n={m}: {np.mean(v):.2f} s x {len(v)}" for m, v in sorted(times.items()))
    sample = (f"oracle Fisher-BT iterations on seeded subsamples, one per step ({meas}), {rule} and "
              f"evaluated at n = {w.n}: {t_full:.0f} s per iteration")
    # ms_per_step is the measured time of a step (a subsample iteration); value is the fitted
    # rate at the full workload, the native arm's unit
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "n": w.n, "theta0": w.theta0},
            "extrapolated_s_per_iteration": t_full,
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def fp64_dmma_peak_tflops():
    """FP64 matrix-multiply rate of this GPU (torch.matmul on float64, the vendor library's DGEMM),
    the denominator of the Cholesky's "% of FP64 tensor peak"; best of 5 at 8192^3."""
    import torch
    a = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    b = torch.randn(8192, 8192, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * 8192 ** 3 / (best * 1e-3) / 1e12


def timed_steps(fbt, ctx, st0, steps, stream):
    """`steps` Fisher-BT iterations from the state st0 (each from st0), timed with CUDA events on
    the context's stream; returns (ms, evaluations, last state)."""
    import torch

    def one_step():
        st = fbt.FbtState()
        ctypes.memmove(ctypes.byref(st), ctypes.byref(st0), ctypes.sizeof(st0))
        fbt.fisher_bt_step(ctx, st)
        return st

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    evals, st = 0, None
    for _ in range(steps):
        st = one_step()
        evals += st.n_ll - st0.n_ll
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), evals, st


def profiled_step(fbt, ctx, st0):
    """One Fisher-BT iteration with the library's per-kernel CUDA-event profiler (graphs off)."""
    st = fbt.FbtState()
    ctypes.memmove(ctypes.byref(st), ctypes.byref(st0), ctypes.sizeof(st0))
    fbt.fbt_profile(ctx, True)
    fbt.fisher_bt_step(ctx, st)
    prof = fbt.fbt_profile_read(ctx)
    fbt.fbt_profile(ctx, False)
    return prof


def run_native(args):
    import torch
    import paper_2601_11437_gb300 as fbt
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    w, locs, z = load_field(args.workload)
    stream = torch.cuda.current_stream(local)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}

    # ---- the value: FP64-accurate path, profiler off, graph replay on ----
    ctx = fbt.fbt_create(locs, z, nb=args.nb, device=local, precision=fbt.PREC_FP64_EMULATED)
    st0 = fbt.fisher_bt_start(ctx, theta0=w.theta0)
    if st0.state != fbt.RUNNING:
        raise RuntimeError(f"start state {st0.state}")
    timed_steps(fbt, ctx, st0, args.warmup, stream)
    clocks = Clocks(local)
    barrier(world, local)
    torch.cuda.synchronize()
    fbt.fbt_launch_count(ctx, reset=True)
    clocks.start()
    ms, evals, _ = timed_steps(fbt, ctx, st0, args.steps, stream)
    ck = clocks.stop()
    launches = fbt.fbt_launch_count(ctx)
    barrier(world, local)
    ms = max_over_ranks(world, ms, local)
    value = world * args.steps / (ms / 1e3)

    # ---- kernel shares and the dominant kernel's per-launch rate: a separate profiled step ----
    prof = profiled_step(fbt, ctx, st0)
    gem = {k: v for k, v in prof.items() if k.startswith("ozaki") and k != "ozaki_slice"}
    dom = max(gem, key=lambda k: gem[k]["ms"])
    per_launch_flops = gem[dom]["flops"] / gem[dom]["launches"]
    per_launch_ms = gem[dom]["ms"] / gem[dom]["launches"]
    fp64eq = per_launch_flops / (per_launch_ms * 1e-3) / 1e12
    bf16_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    achieved = fp64eq * OZAKI_PRODUCTS
    tasks_per_launch = per_launch_flops / OZAKI_TASK_FLOPS
    roof = {"bound": "tensor", "kernel": f"k_ozaki_gemm ({dom})", "achieved": achieved, "peak": bf16_peak,
            "unit": "TFLOP/s", "frac": achieved / bf16_peak,
            "traffic": None if OZAKI_DRAM_BYTES_PER_TASK is None else OZAKI_DRAM_BYTES_PER_TASK * tasks_per_launch,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of this family at "
                               "n = 4096, per task, times this launch's tasks"
                               if OZAKI_DRAM_BYTES_PER_TASK is not None else "no capture of the current kernel"),
            "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained" if "bf16_tflops_sustained" in peaks
                            else "fallback 1.7 PFLOP/s sustained") + " (of measured)",
            "work": "28 BF16 digit products per FP64-accurate tile product",
            "per_launch_ms": per_launch_ms, "tasks_per_launch": tasks_per_launch,
            "fp64_equivalent_tflops": fp64eq}
    total_ms = sum(v["ms"] for v in prof.values())
    # the Cholesky: n^3 / 3 per factorisation over its critical path on the main stream (the
    # diagonal tiles are factored and inverted on a side stream beside the trailing updates)
    chol_fams = ("ozaki_potrf_panel", "ozaki_potrf_update", "cholesky_slice")
    chol_ms = sum(prof[k]["ms"] for k in chol_fams if k in prof)
    n_chol = prof["potrf_diag"]["launches"] / ((w.n + args.nb - 1) // args.nb) if "potrf_diag" in prof else 0
    chol_tf = n_chol * (w.n ** 3 / 3) / (chol_ms * 1e-3) / 1e12 if chol_ms > 0 else None
    dmma = fp64_dmma_peak_tflops()
    cholesky = {"tflops_fp64_equivalent": chol_tf, "ms_per_factorisation": chol_ms / max(n_chol, 1),
                "fp64_matmul_peak_tflops_measured": dmma,
                "frac_of_fp64_matmul_peak": chol_tf / dmma if chol_tf else None,
                "bf16_bound_fp64_equivalent_tflops": bf16_peak / OZAKI_PRODUCTS,
                "frac_of_bf16_bound": chol_tf / (bf16_peak / OZAKI_PRODUCTS) if chol_tf else None,
                "note": "n^3/3 over the summed device time of the factorisation's main-stream kernels "
                        "(profiled step); FP64 matmul peak: torch.matmul float64 8192^3 on this GPU"}

    # ---- the mixed path: same workload and start, fewer steps ----
    mixed = None
    if not args.no_mixed:
        cm = fbt.fbt_create(locs, z, nb=args.nb, device=local, precision=fbt.PREC_MIXED, mixed_tol=args.mixed_tol)
        stm0 = fbt.fisher_bt_start(cm, theta0=w.theta0)
        km = max(1, min(args.steps, args.mixed_steps))
        timed_steps(fbt, cm, stm0, min(args.warmup, 3), stream)
        fbt.fbt_mixed_counts(cm, reset=True)
        ms_m, evals_m, st_m = timed_steps(fbt, cm, stm0, km, stream)
        tiers = fbt.fbt_mixed_counts(cm, reset=True)
        ms_m = max_over_ranks(world, ms_m, local)
        mixed = {"mixed_tol": args.mixed_tol, "steps": km, "warmup": min(args.warmup, 3),
                 "iters_per_s": world * km / (ms_m / 1e3), "ms_per_step": ms_m / km,
                 "speedup_vs_fp64_accurate": (world * km / (ms_m / 1e3)) / value,
                 "evaluations_per_step": evals_m / km,
                 "tile_tasks_per_step": {k: v / km for k, v in tiers.items()},
                 "start_rel_err_vs_fp64_accurate": {
                     "loglik": abs(stm0.loglik - st0.loglik) / abs(st0.loglik),
                     "score": (np.abs(np.array(stm0.score[:]) - np.array(st0.score[:]))
                               / np.abs(np.array(st0.score[:]))).tolist(),
                     "fisher": (np.abs(np.array(stm0.fisher[:]) - np.array(st0.fisher[:]))
                                / np.abs(np.array(st0.fisher[:]))).tolist()}}
        if not args.no_fit:
            # matched theta_hat: Algorithm 1 from theta^(0) on both paths (wall clock, one each)
            fits = {}
            for name, c in (("fp64_accurate", ctx), ("mixed", cm)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fs = fbt.fisher_bt_run(c, theta0=w.theta0)
                torch.cuda.synchronize()
                fits[name] = {"seconds": time.perf_counter() - t0, "theta_hat": list(fs.theta), "state": fs.state,
                              "iterations": fs.iter, "n_ll": fs.n_ll, "n_grad": fs.n_grad,
                              "grad_norm": float(np.linalg.norm(fs.score[:])), "loglik": fs.loglik}
                if name == "mixed":
                    fits[name].update(polish_iter=fs.polish_iter, theta_at_switch=list(fs.theta_mixed))
            th = np.array(fits["fp64_accurate"]["theta_hat"])
            rel = lambda v: float(np.max(np.abs(np.array(v) - th) / np.abs(th)))  # noqa: E731
            mixed["fit"] = fits
            mixed["theta_hat_rel_err"] = rel(fits["mixed"]["theta_hat"])
            mixed["theta_at_switch_rel_err"] = rel(fits["mixed"]["theta_at_switch"])
            mixed["time_to_theta_hat_speedup"] = fits["fp64_accurate"]["seconds"] / fits["mixed"]["seconds"]
        fbt.fbt_destroy(cm)

    # ---- end to end: every step re-creates the context from pinned host buffers (locations and
    # field copied host-to-device), runs the iteration and reads its results back ----
    e2e = None
    if not args.no_e2e:
        pl = torch.from_numpy(np.ascontiguousarray(locs)).pin_memory()
        pz = torch.from_numpy(np.ascontiguousarray(z)).pin_memory()
        ws = ctx.workspace
        fbt.fbt_destroy(ctx)
        lib = fbt._lib.load()
        opts = fbt.FbtOpts()
        lib.fbt_default_opts(ctypes.byref(opts))
        opts.nb, opts.device, opts.precision = args.nb, local, fbt.PREC_FP64_EMULATED
        nbytes = lib.fbt_workspace_bytes(w.n, ctypes.byref(opts))
        wsp = ctypes.c_void_p((ws.data_ptr() + 255) & ~255)
        h2d = d2h = 0
        barrier(world, local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h = ctypes.c_void_p()
            s_ = lib.fbt_create(ctypes.byref(h), ctypes.c_void_p(pl.data_ptr()), 0, ctypes.c_void_p(pz.data_ptr()), 0,
                                w.n, ctypes.byref(opts), wsp, nbytes, ctypes.c_void_p(stream.cuda_stream))
            if s_ != 0:
                raise RuntimeError(f"fbt_create {s_}")
            c = fbt.Context(h.value, w.n, ws, opts)
            st = fbt.FbtState()
            ctypes.memmove(ctypes.byref(st), ctypes.byref(st0), ctypes.sizeof(st0))
            fbt.fisher_bt_step(c, st)
            hb, db = fbt.fbt_transfer_bytes(c)
            h2d += hb
            d2h += db
            fbt.fbt_destroy(c)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(world, time.perf_counter() - t0, local)
        e2e = {"value": world * args.e2e_steps / t_e2e, "unit": "iters/s",
               "h2d_bytes_per_step": h2d // args.e2e_steps, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "steps": args.e2e_steps}
    else:
        fbt.fbt_destroy(ctx)

    if rank != 0:
        return 0
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(locs, z, w)
    slab_gb = 3 * 8.0 * ((w.n + args.nb - 1) // args.nb) ** 2 * args.nb ** 2 / 2 / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "nb": args.nb, "theta_true": w.theta_true,
                   "theta0": w.theta0, "jitter": w.jitter, "parallelism": f"replicas{world}",
                   "value_path": "FP64-accurate tile updates from exact BF16 digit products on tcgen05 tensor "
                                 "cores (7 x 8-bit balanced slices, FP32 TMEM groups, FP64 recombination); "
                                 "all else FP64; profiler off, graph replay on",
                   "evaluations_per_step": evals / args.steps,
                   "l2": f"no flush: each step streams 3 x {slab_gb / 3:.1f} GB of tile slabs, far above the 129 MB L2"},
        "mixed": mixed,
        "cholesky": cholesky,
        "roofline": roof,
        "fp64_peak_tflops": FP64_PEAK_TFLOPS,
        "kernel_share": {k: round(v["ms"] / total_ms, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
        "kernel_share_note": "shares of the summed family times of one profiled step (taken after the timed region); "
                             "potrf_diag and trtri_panel run on a side stream, mostly overlapped",
        "gpu_launches": launches,
        "clocks": ck,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


def load_batch(name: str):
    """The stored batched-fields workload: per-field recipe, locations and z."""
    meta = json.load(open(os.path.join(FIELDS, f"{name}_z.json")))
    fl = inputs.batched_fields(meta["fields"])
    zall = np.load(os.path.join(FIELDS, f"{name}_z.npy"))
    h, out, o = hashlib.sha256(), [], 0
    for f in fl:
        locs = inputs.uniform_locations(f.n, f.seed)
        h.update(np.ascontiguousarray(locs, dtype="<f8").tobytes())
        out.append((f, locs, zall[o:o + f.n]))
        o += f.n
    if h.hexdigest() != meta["locations_sha256"] or o != zall.size:
        raise RuntimeError(f"stored batch {name} does not belong to these locations")
    return out


def run_batch(args):
    """Batched independent fields: a step is one Fisher-BT iteration of every field, all fields
    driven concurrently (host thread pool, one stream per thread), each from its theta^(0) state."""
    import torch
    import paper_2601_11437_gb300 as fbt
    from paper_2601_11437_gb300 import sharding
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    full = load_batch(args.workload)
    # N > 1: the fields are independent units, shared out by cost; no exchange until the end
    mine = sharding.partition([f.n ** 3 for f, _, _ in full], world)[rank]
    batch = [full[i] for i in mine]
    prec = PRECISIONS[args.precision]
    theta0s = np.array([f.theta0 for f, _, _ in batch])
    tuning = None
    if args.autotune and args.precision in ("fp64", "fp64_emulated"):
        # per size band (n rounded up to a power of two) the faster FP64-accurate configuration,
        # measured on the band's first field; then the host-thread count over the whole batch
        choice, bands = {}, {}
        for f, locs, z in batch:
            band = 1 << (f.n - 1).bit_length()
            if band not in choice:
                p_, nb_, secs, _ = fbt.fbt_autotune(locs, z, f.theta0, precision=prec, device=local)
                choice[band] = (p_, nb_)
                bands[str(band)] = {"precision": {v: k for k, v in PRECISIONS.items()}[p_], "nb": nb_,
                                    "seconds_per_eval": secs}
        ctxs = []
        for f, locs, z in batch:
            p_, nb_ = choice[1 << (f.n - 1).bit_length()]
            ctxs.append(fbt.fbt_create(locs, z, nb=nb_, device=local, precision=p_))
        best, secs = fbt.fbt_tune_batch_threads(ctxs, theta0s, candidates=(8, 16, 32, 64))
        args.threads = best
        tuning = {"bands": bands, "threads": best, "threads_seconds_per_pass": secs,
                  "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")}
    else:
        ctxs = [fbt.fbt_create(locs, z, nb=args.nb, device=local, precision=prec) for _, locs, z in batch]
    st0, status = fbt.fisher_bt_start_batch(ctxs, theta0s, nthreads=args.threads)
    running = [q for q in range(len(ctxs)) if st0[q].state == fbt.RUNNING]
    run_ctxs = [ctxs[q] for q in running]
    ns = np.array([batch[q][0].n for q in running], dtype=np.float64)

    def one_step():
        st = (fbt.FbtState * len(running))()
        for i, q in enumerate(running):
            ctypes.memmove(ctypes.byref(st[i]), ctypes.byref(st0[q]), ctypes.sizeof(fbt.FbtState))
        fbt.fisher_bt_step_batch(run_ctxs, st, nthreads=args.threads)
        return st

    for _ in range(args.warmup):
        one_step()
    for c in run_ctxs:
        fbt.fbt_launch_count(c, reset=True)
    clocks = Clocks(local)
    barrier(world, local)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    flops = 0.0
    for _ in range(args.steps):
        st = one_step()
        for i, q in enumerate(running):
            lls = st[i].n_ll - st0[q].n_ll - (st[i].n_grad - st0[q].n_grad)
            flops += lls * ns[i] ** 3 / 3 + (st[i].n_grad - st0[q].n_grad) * 7 * ns[i] ** 3 / 3
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ck = clocks.stop()
    barrier(world, local)
    sec = max_over_ranks(world, sec, local)
    launches = sum(fbt.fbt_launch_count(c) for c in run_ctxs)
    for c in ctxs:
        fbt.fbt_destroy(c)
    n_stepped = len(running)
    if world > 1:
        # the one exchange: every field's 13-double record of its last step, gathered in field order
        import torch.distributed as dist
        g = dist.new_group(backend="gloo")
        pos = {q: i for i, q in enumerate(running)}
        recs = []
        for q in range(len(batch)):                 # fields that did not step report their start
            s_ = st[pos[q]] if q in pos else st0[q]
            recs.append([s_.loglik, *s_.score[:], *s_.fisher[:]])
        sharding.gather_records(mine, recs, len(full), group=g)
        tot = torch.tensor([float(n_stepped), flops, float(launches)], dtype=torch.float64, device=f"cuda:{local}")
        dist.all_reduce(tot)
        n_stepped, flops, launches = int(tot[0].item()), float(tot[1].item()), int(tot[2].item())
    if rank != 0:
        return 0
    line = {
        "metric": "fields x Fisher-BT iterations/s (batched fields)", "value": n_stepped * args.steps / sec,
        "unit": "field-iters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "fields": len(full), "fields_stepped": n_stepped,
                   "parallelism": f"fields sharded over {world} rank(s) by n^3, records gathered",
                   "n_range": [min(f.n for f, _, _ in full), max(f.n for f, _, _ in full)],
                   "sum_n3": float(sum(float(f.n) ** 3 for f, _, _ in full)),
                   "precision": args.precision, "threads": args.threads, "nb": args.nb, "autotune": tuning,
                   "timing": "host wall clock around each batched call (it synchronises every stream)"},
        "aggregate_tflops_fp64_equivalent": flops / sec / 1e12,
        "gpu_launches": launches, "clocks": ck, "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args):
    """Adjoint gradient at theta_true: forward l (Algorithm 2), backward (adjoint), the Fisher path's
    score and central finite differences of l, on one large field."""
    import torch
    import paper_2601_11437_gb300 as fbt
    w, locs, z = load_field(args.workload)
    ctx = fbt.fbt_create(locs, z, nb=128, precision=PRECISIONS[args.precision])
    th = np.array(w.theta_true)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(args.warmup):
        fbt.mle_loglik(ctx, th * 1.01)
        fbt.mle_loglik_grad(ctx, th * 1.01)
    fwd, bwd = [], []
    for _ in range(args.steps):
        fbt.mle_loglik(ctx, th * 1.02)                    # a different point: the next forward factorises
        ev[0].record(stream)
        ll = fbt.mle_loglik(ctx, th)
        ev[1].record(stream)
        ll_g, g = fbt.mle_loglik_grad(ctx, th)            # reuses the forward's factor
        ev[2].record(stream)
        torch.cuda.synchronize()
        fwd.append(ev[0].elapsed_time(ev[1]))
        bwd.append(ev[1].elapsed_time(ev[2]))
    ev[0].record(stream)
    ll_e, g_e, _ = fbt.mle_eval(ctx, th)
    ev[1].record(stream)
    torch.cuda.synchronize()
    eval_ms = ev[0].elapsed_time(ev[1])
    # fourth-order central differences, h = 1e-3 theta_i: truncation ~h^4, and l's evaluation
    # noise (~1e-11 relative at this size) enters as ~1e-11 |l| / h
    fd = np.empty(3)
    for i in range(3):
        h = 1e-3 * th[i]
        f = {}
        for s_ in (-2, -1, 1, 2):
            t = th.copy()
            t[i] += s_ * h
            f[s_] = fbt.mle_loglik(ctx, t)
        fd[i] = (8 * (f[1] - f[-1]) - (f[2] - f[-2])) / (12 * h)
    fbt.fbt_destroy(ctx)
    n = w.n
    line = {
        "metric": "adjoint backward time (s)", "value": statistics.median(bwd) / 1e3, "unit": "s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": n, "theta": w.theta_true, "precision": args.precision},
        "forward_s": statistics.median(fwd) / 1e3, "mle_eval_s": eval_ms / 1e3,
        "backward_tflops_fp64_equivalent": (2 * n ** 3 / 3) / (statistics.median(bwd) * 1e-3) / 1e12,
        "loglik": ll, "grad": g.tolist(), "score_fisher_path": g_e.tolist(), "grad_central_fd": fd.tolist(),
        "rel_err_vs_fisher_path": float(np.abs(g - g_e).max() / np.abs(g_e).max()),
        "rel_err_vs_fd": float(np.abs(g - fd).max() / np.abs(g).max()),
        "loglik_equal": bool(ll == ll_g == ll_e),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_compare(args):
    """Mixed against emulated FP64 on one large field: l, score, Fisher at theta^(0), the Cholesky
    rate, and the Fisher-BT estimate of each path (Algorithm 1 to convergence)."""
    import torch
    import paper_2601_11437_gb300 as fbt
    w, locs, z = load_field(args.workload)
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec in (("fp64_emulated", fbt.PREC_FP64_EMULATED), ("mixed", fbt.PREC_MIXED)):
        ctx = fbt.fbt_create(locs, z, nb=128, precision=prec)
        fbt.mle_loglik(ctx, np.array(w.theta0) * 1.01)             # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fbt.fbt_profile(ctx, True)
        ev[0].record(stream)
        fbt.mle_loglik(ctx, w.theta0)
        ev[1].record(stream)
        ll, g, I = fbt.mle_eval(ctx, w.theta0)                      # reuses the factor
        ev[2].record(stream)
        torch.cuda.synchronize()
        prof = fbt.fbt_profile_read(ctx)
        fbt.fbt_profile(ctx, False)
        chol = {k: v for k, v in prof.items() if k in ("potrf_diag", "trsm_panel", "trtri_panel", "ozaki_potrf_panel",
                                                       "ozaki_potrf_update", "ozaki_slice")}
        # the slicing of the Cholesky's panels is counted with the Cholesky (the transforms' slices are not)
        chol_ms = sum(v["ms"] for k, v in chol.items() if k != "ozaki_slice")
        n = w.n
        t0 = time.perf_counter()
        st = fbt.fisher_bt_run(ctx, theta0=w.theta0)
        torch.cuda.synchronize()
        fit_s = time.perf_counter() - t0
        out[name] = {"loglik_s": ev[0].elapsed_time(ev[1]) / 1e3, "mle_eval_s": ev[1].elapsed_time(ev[2]) / 1e3,
                     "cholesky_tflops_fp64_equivalent": (n ** 3 / 3) / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e12,
                     "cholesky_kernel_ms": chol_ms,
                     "loglik": ll, "score": g.tolist(), "fisher": I.tolist(),
                     "theta_hat": list(st.theta), "state": st.state, "iterations": st.iter,
                     "n_ll": st.n_ll, "n_grad": st.n_grad, "fit_s": fit_s,
                     "fisher_bt_iters_per_s": st.iter / fit_s if st.iter else None}
        fbt.fbt_destroy(ctx)
    e, m = out["fp64_emulated"], out["mixed"]
    rel = lambda a, b: float(np.max(np.abs(np.array(a) - np.array(b))) / np.max(np.abs(np.array(b))))  # noqa: E731
    line = {"metric": "mixed vs FP64-accurate path", "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "theta0": w.theta0, "theta_true": w.theta_true,
                       "mixed_tol": 1e-12},
            "rel_err_loglik": abs(m["loglik"] - e["loglik"]) / abs(e["loglik"]),
            "rel_err_score": rel(m["score"], e["score"]), "rel_err_fisher": rel(m["fisher"], e["fisher"]),
            "rel_err_theta_hat": rel(m["theta_hat"], e["theta_hat"]),
            "speedup_mle_eval": e["mle_eval_s"] / m["mle_eval_s"], "speedup_loglik": e["loglik_s"] / m["loglik_s"],
            "paths": out}
    print(json.dumps(line), flush=True)
    return 0


def run_sim(args):
    """The simulation study (Sec. 3): every stored realisation of every (setting, n) fitted by
    Algorithm 1 from the L9 design over the study's box, realisations of one (setting, n) as one
    batch; per (setting, n) the estimates' mean and spread, the microergodic theta_m =
    sigma^2 alpha^(-2 nu), iterations, l and derivative calls, Nelder-Mead shifts and time."""
    import torch
    import paper_2601_11437_gb300 as fbt
    meta = json.load(open(os.path.join(FIELDS, f"{args.workload}_z.json")))
    zall = np.load(os.path.join(FIELDS, f"{args.workload}_z.npy"))
    reps = meta["reps"]
    prec = PRECISIONS[args.precision]
    lo, hi = np.array(inputs.SIM_BOX[0]), np.array(inputs.SIM_BOX[1])
    h, o, rows = hashlib.sha256(), 0, []
    t_all = time.perf_counter()
    for n in inputs.SIM_SIZES:
        locs = inputs.sim_locations(n)
        h.update(np.ascontiguousarray(locs, dtype="<f8").tobytes())
        for si, th in enumerate(inputs.SIM_SETTINGS):
            zs = [zall[o + r * n:o + (r + 1) * n] for r in range(reps)]
            o += reps * n
            ctxs = [fbt.fbt_create(locs, z, nb=args.nb, precision=prec) for z in zs]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            states, status = fbt.fisher_bt_run_batch(ctxs, theta_lo=np.tile(lo, (reps, 1)),
                                                     theta_hi=np.tile(hi, (reps, 1)), nthreads=args.threads)
            dt = time.perf_counter() - t0
            for c in ctxs:
                fbt.fbt_destroy(c)
            est = np.array([list(st.theta) for st in states])
            tm = est[:, 0] * est[:, 1] ** (-2 * est[:, 2])
            rows.append({
                "n": n, "theta_true": th, "theta_m_true": th[0] * th[1] ** (-2 * th[2]),
                "theta_hat_mean": est.mean(0).round(6).tolist(), "theta_hat_sd": est.std(0, ddof=1).round(6).tolist(),
                "theta_m_mean": float(np.mean(tm)), "theta_m_sd": float(np.std(tm, ddof=1)),
                "iterations_mean": float(np.mean([st.iter for st in states])),
                "l_calls_mean": float(np.mean([st.n_ll for st in states])),
                "derivative_calls_mean": float(np.mean([st.n_grad for st in states])),
                "nelder_mead_fraction": float(np.mean([st.state == fbt.DONE_NM for st in states])),
                "failed": int(np.sum([(st.state == fbt.FAILED) or s_ != fbt.FBT_OK for st, s_ in zip(states, status)])),
                "seconds_per_fit_in_batch": dt / reps, "batch_seconds": dt})
    if h.hexdigest() != meta["locations_sha256"] or o != zall.size:
        raise RuntimeError(f"stored {args.workload} does not belong to these designs")
    line = {"metric": "simulation study (Sec. 3): Fisher-BT fits from the L9 design", "n_gpus": 1,
            "dtype": "f64", "data": "synthetic", "precision": args.precision, "reps": reps,
            "box": inputs.SIM_BOX, "total_seconds": time.perf_counter() - t_all, "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_single_eval(args):
    """One Algorithm 3 evaluation at theta^(0) (generation, Cholesky, transforms), nothing else:
    the target of kernel captures on a small case.  FP64-accurate unless --precision mixed, which
    runs the mixed path at --mixed-tol."""
    import torch
    import paper_2601_11437_gb300 as fbt
    w, locs, z = load_field(args.workload)
    if args.precision == "mixed":
        ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_MIXED, mixed_tol=args.mixed_tol)
    else:
        ctx = fbt.fbt_create(locs, z, nb=128, precision=fbt.PREC_FP64_EMULATED)
    ll, g, I = fbt.mle_eval(ctx, w.theta0)
    torch.cuda.synchronize()
    fbt.fbt_destroy(ctx)
    print(json.dumps({"workload": w.name, "n": w.n, "loglik": ll, "score": g.tolist()}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="n65536")
    ap.add_argument("--nb", type=int, default=128)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp64_emulated")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-sizes", type=lambda v: [int(x) for x in v.split(",")],
                    default=list(ORACLE_SIZES), help="oracle subsample sizes of the reference arm")
    ap.add_argument("--mixed-tol", type=float, default=1e-6,
                    help="tolerance of the mixed path's line entry (1e-6: the loosest whose estimate at the "
                         "switch meets the 1e-3 criterion at n = 65,536)")
    ap.add_argument("--mixed-steps", type=int, default=5, help="timed steps of the mixed path (at most --steps)")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-fit", action="store_true", help="skip the two Fisher-BT fits (matched theta_hat)")
    ap.add_argument("--threads", type=int, default=16, help="host threads of the batched workload")
    ap.add_argument("--autotune", action="store_true",
                    help="batched workload: tune the FP64-accurate configuration per size band and the thread count")
    ap.add_argument("--adjoint", action="store_true", help="time the adjoint gradient on --workload")
    ap.add_argument("--single-eval", action="store_true",
                    help="one Algorithm 3 evaluation on --workload (a kernel-capture target; FP64-accurate "
                         "unless --precision mixed)")
    ap.add_argument("--compare-mixed", action="store_true",
                    help="mixed against emulated FP64 on --workload (errors, Cholesky rate, estimates)")
    args = ap.parse_args()
    if args.workload.startswith("batch") and args.impl == "native":
        return run_batch(args)
    if args.workload.startswith("sim") and args.impl == "native":
        return run_sim(args)
    if args.single_eval:
        return run_single_eval(args)
    if args.adjoint:
        return run_adjoint(args)
    if args.compare_mixed:
        return run_compare(args)
    if args.precision != "fp64_emulated" and args.impl == "native":
        # the single-field line measures the FP64-accurate path with the mixed path beside it
        ap.error("--precision applies to the batched, simulation and adjoint modes; the single-field line "
                 "always measures the FP64-accurate path with the mixed path (--mixed-tol) beside it, "
                 "and --compare-mixed compares the two in detail")
    if args.warmup < 3 and args.impl == "native" and not os.environ.get("FBT_BENCH_ALLOW_SHORT"):
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    return run_reference(args) if args.impl == "reference" else run_native(args)


if __name__ == "__main__":
    sys.exit(main())
