#!/usr/bin/env python
"""Benchmark of the octree-block multigrid solve on GB300 (one JSON line on stdout, rank 0).

Workload (default 'uniform_8x64_k'): 8^3 root blocks of 64^3 cells (512^3 = 134,217,728 cells) on the unit cube,
-div(k grad u) = f with k = exp(g), g a seeded Gaussian random field (sigma 1, correlation length 0.1, random
Fourier features), f ~ U(-1, 1) seeded, homogeneous Dirichlet data.  One step = one solve from u = 0 to a 1e-10
relative residual with FP32 V(2,2) cycles inside FP64 defect correction (every kernel of the path runs: ghost
exchange, red-black Gauss-Seidel, residual + restriction, prolongation, dense coarsest solve, FP64 outer residual
and update).  The plain FP64 V-cycle solve of the same problem is timed in the same run.

Metric: GLUPS per V(2,2) cycle = cells x cycles / time / 1e9, summed over ranks (independent replicas: the
solver does not shard across GPUs).  Inputs (~4 GB per replica) exceed the 129 MB L2, so no flush is needed.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "GLUPS per V(2,2) cycle (FP32-in-FP64 solve to 1e-10 relative residual)"
UNIT = "GLUPS"

WORKLOADS = {
    # name: (forest, coefficient, rhs)
    "uniform_8x64_k": ("uniform_8x64", True, "uniform"),
    "sphere_2x32": ("sphere_2x32", False, "bump"),
    "uniform_4x64_k": ("uniform_4x64", True, "uniform"),
    "batch_256": ("batch", True, "uniform"),   # 256 single-root problems, n in {16,32,64,128}, 0-2 box refinements
    "batch_32": ("batch", True, "uniform"),    # 32 such problems (smaller case of the same recipe)
    # the paper's own experiments (Sec. 5 and 6), FP64 with its V(3,3) damped-Jacobi cycle
    "paper_bench": ("paper_bench", False, "uniform"),  # 22 R^3 blocks of 64^3 (R = 4: 1408 blocks), 100 cycles
    "paper_table": ("sphere", False, "zero"),           # Table err_analysis: errors for block sizes 16 .. 128
}


def _inputs(workload, device, seed=0):
    import synthetic as syn
    forest, coeff, rhs = WORKLOADS[workload]
    R, n, keys = syn.workload_forest(forest)
    k = syn.lognormal_k_rff(R, n, keys, seed=seed, device=device) if coeff else None
    if rhs == "uniform":
        f = syn.uniform_rhs(len(keys), n, seed=seed + 1).to(device)
    else:
        f = syn.gaussian_bump_with_noise(R, n, keys, seed=seed + 1, device=device)
    return R, n, keys, k, f


# ------------------------------------------------------------------------------------------------------------
# byte and flop models of the kernel families (per cell of the level a launch covers)
# ------------------------------------------------------------------------------------------------------------
def _family_work(fam, levels, nu1, nu2, coeff, cycles_total, outer_total, launches=0):
    """Algorithmic bytes and FP64 flops of one family over the timed region.

    Per cell of the level a launch sweeps:
      smooth_f32       8 B   (half of a full red-black iteration's u, f, k read and u written, 4 B each; 6 B for
                             constant k.  The two-launch schedule itself moves 10 B: see _SCHEDULE_BYTES_HALF_SWEEP)
      smooth_f64      12 B   (24 B/cell RBGS iteration for -Laplace in FP64: u, f, u)
      residual_f64    32 B   (u, f, k read as FP64; r written as FP32; FP32 correction zeroed) and 27 FP64 flops
                             (stencil 11, diagonal 5, residual 4, scaling 1, two volume-weighted norms 6)
      update_mixed    20 B   (u64 read + write, e32 read)
    """
    cells = [nb * n ** 3 for nb, n in levels]
    sweeps = 2 * (nu1 + nu2)
    f32b = _ALG_BYTES_HALF_SWEEP[bool(coeff)]
    if fam == "smooth_f32_finest":
        return cells[0] * f32b * launches, 0.0
    if fam == "smooth_f64_finest":
        return cells[0] * (16 if coeff else 12) * launches, 0.0
    if fam == "smooth_f32":
        b = sum(c for c in cells[:-1]) * sweeps * f32b * cycles_total
        return b, 0.0
    if fam == "smooth_f64":
        per = 16 if coeff else 12
        b = sum(c for c in cells[:-1]) * sweeps * per * cycles_total
        return b, 0.0
    if fam == "residual_f64":
        return cells[0] * 32 * outer_total, cells[0] * 27.0 * outer_total
    if fam == "update_mixed":
        return cells[0] * 20 * launches, 0.0
    return None, None


# DRAM bytes per cell of the level per launch, from one ncu capture of the kernel on the 16.8M-cell case
# (dram__bytes_read.sum + dram__bytes_write.sum divided by the level's cells), scaled here to the launch's cells
# (the traffic grows in proportion to the cells).
_NCU_TRAFFIC_PER_CELL = {
    "smooth_f32_finest": (164.37632e6 / 16777216, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                          "k_smooth32t<2,6,4> launch (rows in pairs, colour-reversed tile order), shape {2,16,16,4,4}, "
                          "on 4^3 roots of 64^3 cells (16,777,216 cells, log-normal k), scaled by cells"),
}

# Algorithmic bytes of the FP32 red-black smoother per cell: a full iteration reads u, f and k and writes u once,
# 4 B each, 16 B per cell (12 B with constant k), i.e. 8 (6) B per one-colour launch.  The two-launch schedule moves
# 10 B per launch with variable k (the other colour's u, this colour's f, both colours' 1/k, this colour's u written)
# and the same 6 B with constant k.
_ALG_BYTES_HALF_SWEEP = {True: 8.0, False: 6.0}
_SCHEDULE_BYTES_HALF_SWEEP = {True: 10.0, False: 6.0}
# Bytes per finest cell per V(2,2) cycle (FP32 cycles, variable k, levels summed with the 8/7 geometric factor):
# the unfused model with one FP64 outer residual per cycle, and the minimum of one fused down- and up-pass per level.
_CYCLE_BYTES_MIXED = 78.0
_CYCLE_BYTES_ALG_MIN = 37.7
# face-averaged coarse levels read three FP32 face arrays instead of one 1/k: +8 B per coarse cell in each of the four
# smoother passes and in the residual + restriction, 40 B per coarse cell and cycle, 1/7 coarse cell per finest cell
_CYCLE_BYTES_FACES_EXTRA = 40.0 / 7.0

HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal

_COARSE_COEF_NAMES = {"faces": "face-averaged from the finer level", "k": "rediscretised from the children's mean k"}


def _smoother_report(prof, cells):
    """Finest-level FP32 smoother throughput in the paper's per-kernel sense: finest cells x full sweeps / smoother
    time, from the profiled pass (each launch is one colour's half-sweep over the whole finest level)."""
    ms, launches = prof.get("smooth_f32_finest", (0.0, 0))
    if launches < 2 or ms <= 0.0:
        return None
    return {"glups": cells * (launches // 2) / (ms / 1e3) / 1e9, "sweeps": launches // 2, "ms": round(ms, 3)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mp = json.load(fh)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            bus = torch.cuda.get_device_properties(self.dev).pci_bus_id if hasattr(
                torch.cuda.get_device_properties(self.dev), "pci_bus_id") else None
        except Exception:
            bus = None
        sel = ["-i", bus] if bus else []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", *sel], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    """(torch.distributed or None, rank, world size, local rank) from the torchrun environment.  Ranks are
    independent replicas: the process group only carries the barriers and the max-over-ranks of the timings (NCCL
    with GPUs, gloo without)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
        return dist, rank, ws, local
    return None, 0, 1, 0


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, x):
    if dist is None:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline): bounded sample of the same recipe
# ------------------------------------------------------------------------------------------------------------
ORACLE_SAMPLE = ("uniform_2x64", "2^3 roots of 64^3 cells (2,097,152 cells) of the same recipe (log-normal k, "
                 "U(-1,1) f), FP64 V(2,2) cycles of the numpy oracle; cores = process CPU time / wall time")


def _host_cpu():
    """The host's logical CPU count and CPU model (/proc/cpuinfo, else lscpu, else the machine name)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith(("model name", "vendor id")):
                    model = (model + " / " if model else "") + line.split(":", 1)[1].strip()
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.machine()}


def _cores(cpu_s, wall_s):
    """Host cores the timed oracle loop kept busy: process CPU time (all threads) over wall time, at least 1."""
    return max(1, round(cpu_s / wall_s))


def _oracle_setup():
    import synthetic as syn
    from oracle.octree_mg import OracleMG
    R, n = 2, 64
    keys = syn.uniform_leaves(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=0).numpy()
    f = syn.uniform_rhs(len(keys), n, seed=1).numpy()
    mg = OracleMG(R, n, keys, k_user=k)
    return mg, f, len(keys) * n ** 3


def _oracle_cycle(mg, f, U, F):
    mg.vcycle(0, U, F)


def run_reference(args):
    dist, rank, ws, _ = _dist()
    if rank != 0:
        return
    mg, f, cells = _oracle_setup()
    F = mg.to_pad(f)[:, 1:-1, 1:-1, 1:-1].copy()
    U = mg.levels[0].zeros()
    for _ in range(args.warmup):
        mg.vcycle(0, U, F)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        mg.vcycle(0, U, F)
    dt = time.perf_counter() - t0
    cores = _cores(time.process_time() - c0, dt)
    value = cells * args.steps / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": ORACLE_SAMPLE[0]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": ORACLE_SAMPLE[1],
                         **_host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(budget_s=12.0):
    """The oracle's FP64 V-cycles on the host, as many as fit in about budget_s seconds (at least two)."""
    mg, f, cells = _oracle_setup()
    F = mg.to_pad(f)[:, 1:-1, 1:-1, 1:-1].copy()
    U = mg.levels[0].zeros()
    n = 0
    t0, c0 = time.perf_counter(), time.process_time()
    while True:
        mg.vcycle(0, U, F)
        n += 1
        if n >= 2 and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = _cores(time.process_time() - c0, dt)
    return {"value": cells * n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{ORACLE_SAMPLE[1]}; {n} cycles in {dt:.1f} s", **_host_cpu()}


# ------------------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------------------
def run_ours(args):
    from paper_2403_08063_gb300 import Forest, alu_peaks
    dist, rank, ws, local = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    R, n, keys, k, f = _inputs(args.workload, dev)
    coeff = k is not None
    cells = len(keys) * n ** 3
    F = Forest(R, n, keys, coeff=coeff, precision=1, inner_cycles=args.inner_cycles, coarse_coef=args.coarse_coef)
    F.set_rhs(f, k)
    if args.tail != "auto":
        F.set_tail(int(args.tail))
    if args.smoother_shape:
        F.set_smoother_shape(0, [int(v) for v in args.smoother_shape.split(",")])
    levels = F.levels()
    u = torch.zeros_like(f)
    alu = alu_peaks()  # measured FP64 / FP32 FMA TFLOP/s (before the timed region; synchronises the device)

    def step(forest):
        u.zero_()
        cyc, rel = forest.solve(u, rtol=args.rtol, max_cycles=60)
        return cyc, rel

    for _ in range(args.warmup):
        step(F)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    _barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("mg_timed")
    e0.record(stream)
    cycles = []
    rels = []
    for _ in range(args.steps):
        c, r = step(F)
        cycles.append(c)
        rels.append(r)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    _barrier(dist)
    # the same K solves again with a CUDA-event pair around every kernel family (the events add a little time, so
    # `value` comes from the run above and the per-family times and the roofline from this one)
    F.profile(True)
    torch.cuda.nvtx.range_push("mg_profiled")
    for _ in range(args.steps):
        step(F)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = F.profile_read()
    F.profile(False)
    t = _max_over_ranks(dist, e0.elapsed_time(e1) / 1e3)
    tot_cycles = sum(cycles)
    value = cells * tot_cycles / t / 1e9 * ws
    launches = sum(v[1] for v in prof.values())

    # roofline of the dominant family; the smoother is reported on its finest-level launches (the coarse levels'
    # launches are separate families), which carry ~88 % of its time
    fam = max((k_ for k_ in prof if prof[k_][1] > 0), key=lambda k_: prof[k_][0] +
              (prof.get("smooth_f32", (0, 0))[0] if k_ == "smooth_f32_finest" else 0.0))
    outer = prof.get("residual_f64", (0, 0))[1] // 2  # k_residual_norm + partial-sum launches per residual
    bytes_, flops = _family_work(fam, levels, 2, 2, coeff, tot_cycles, outer, prof[fam][1])
    hbm, src = _peaks()
    fam_s = prof[fam][0] / 1e3
    roof = None
    if bytes_ is not None:
        if fam == "residual_f64":
            ach = flops / fam_s / 1e12
            roof = {"kernel": fam, "bound": "alu", "achieved": ach, "peak": alu[0], "unit": "TFLOP/s",
                    "frac": ach / alu[0], "traffic": None, "peak_source": "measured FP64 FMA rate (mg_alu_peaks)",
                    "hbm_achieved_gbs": bytes_ / fam_s / 1e9}
        else:
            ach = bytes_ / fam_s / 1e9
            tr = _NCU_TRAFFIC_PER_CELL.get(fam) if args.workload.startswith("uniform") and coeff else None
            roof = {"kernel": fam, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "traffic": tr[0] * levels[0][0] * levels[0][1] ** 3 if tr else None, "peak_source": src,
                    "algorithmic_bytes_per_cell": _ALG_BYTES_HALF_SWEEP[coeff] if fam.startswith("smooth_f32")
                    else None,
                    "frac_of_nominal": ach / HBM_NOMINAL_GBS, "nominal_peak": HBM_NOMINAL_GBS}
            if fam.startswith("smooth_f32"):
                sched = _SCHEDULE_BYTES_HALF_SWEEP[coeff] / _ALG_BYTES_HALF_SWEEP[coeff]
                roof["schedule_bytes_per_cell"] = _SCHEDULE_BYTES_HALF_SWEEP[coeff]
                roof["frac_schedule_bytes"] = ach * sched / hbm
                roof["schedule_over_algorithmic"] = sched
            if tr:
                roof["traffic_source"] = tr[1]
                roof["traffic_bytes_per_cell"] = tr[0]
        roof["launches"] = prof[fam][1]
        roof["avg_launch_ms"] = prof[fam][0] / max(1, prof[fam][1])

    # the FP64 outer residual against the measured FP64 FMA rate (it is bound by FP64 arithmetic, not by HBM)
    res_roof = None
    if prof.get("residual_f64", (0, 0))[1] > 0:
        rb, rfl = _family_work("residual_f64", levels, 2, 2, coeff, tot_cycles, outer)
        rs = prof["residual_f64"][0] / 1e3
        res_roof = {"kernel": "residual_f64", "bound": "alu", "achieved": rfl / rs / 1e12, "peak": alu[0],
                    "unit": "TFLOP/s", "frac": rfl / rs / 1e12 / alu[0], "peak_source": "measured FP64 FMA rate",
                    "flops_per_cell": 27, "hbm_achieved_gbs": rb / rs / 1e9}

    # the set-up alone (mg_set_rhs: coefficient pyramid, coarsest inverse, right-hand side and its norms), kept out of
    # `value`: the first repeat records the coarsest inverse's graph, the second is timed
    F.set_rhs(f, k)
    torch.cuda.synchronize()
    q0 = time.perf_counter()
    F.set_rhs(f, k)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - q0) * 1e3

    # plain FP64 V-cycles on the same problem (time to 1e-10)
    F64 = Forest(R, n, keys, coeff=coeff, precision=0, coarse_coef=args.coarse_coef)
    F64.set_rhs(f, k)
    step(F64)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps64 = 2
    s0.record(stream)
    cyc64 = []
    for _ in range(reps64):
        c, _r = step(F64)
        cyc64.append(c)
    s1.record(stream)
    torch.cuda.synchronize()
    t64 = s0.elapsed_time(s1) / 1e3 / reps64
    F64.close()

    # the other coarse operator on the same problem (time to rtol, both arms), for comparison
    alt = None
    if coeff:
        other = "k" if args.coarse_coef == "faces" else "faces"
        alt = {"coarse_coefficients": _COARSE_COEF_NAMES[other]}
        for name, prec, inner in (("fp32_in_fp64", 1, args.inner_cycles), ("fp64", 0, 1)):
            G = Forest(R, n, keys, coeff=True, precision=prec, inner_cycles=inner, coarse_coef=other)
            G.set_rhs(f, k)
            step(G)
            res, tg = _timed(lambda: step(G), 2)
            alt[name] = {"time_to_rtol_ms": tg * 1e3, "cycles": res[-1][0]}
            G.close()
            del G
        alt["speedup_fp32_in_fp64"] = alt["fp64"]["time_to_rtol_ms"] / alt["fp32_in_fp64"]["time_to_rtol_ms"]

    # end to end through the C ABI with host buffers (mg_solve_host): H2D of f and k, the set-up, the solve from a zero
    # initial guess, D2H of u -- one library call per step, timed on the host around it
    fh = f.cpu().pin_memory()
    kh = k.cpu().pin_memory() if coeff else None
    uh = torch.empty_like(fh).pin_memory()
    F.solve_host(fh, kh, u=uh, rtol=args.rtol, max_cycles=60)  # first call: device staging buffers
    torch.cuda.synchronize()
    _barrier(dist)
    e2e_steps = max(1, args.steps)  # the same K steps as the device-timed value
    e2e_cycles = 0
    h0 = time.perf_counter()
    for _ in range(e2e_steps):
        _u, c, _r = F.solve_host(fh, kh, u=uh, rtol=args.rtol, max_cycles=60)
        e2e_cycles += c
    torch.cuda.synchronize()
    te2e = _max_over_ranks(dist, time.perf_counter() - h0)

    out = None
    if rank == 0:
        tmix = t / args.steps
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 cycles + f64 outer", "data": "synthetic",
            "config": {"workload": args.workload, "cells": cells, "blocks": len(keys), "block": f"{n}^3",
                       "levels": levels, "coefficient": "log-normal k (sigma 1, ell 0.1)" if coeff else "1",
                       "rhs": WORKLOADS[args.workload][2], "rtol": args.rtol, "cycle": "V(2,2) red-black GS",
                       "inner_cycles": args.inner_cycles,
                       "coarse_coefficients": _COARSE_COEF_NAMES[args.coarse_coef] if coeff else None,
                       "smoother_shapes": [list(F.smoother_shape(l)) for l in range(len(levels))],
                       "persistent_tail_from_level": F.tail_level(),
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"{ws} independent replicas"},
            "cycles_per_solve": cycles, "final_rel_residual": rels[-1],
            "time_to_rtol_s": {"fp32_in_fp64": tmix, "fp64": t64, "speedup": t64 / tmix},
            "fp64_cycles_per_solve": cyc64, "fp64_glups_per_cycle": cells * statistics.mean(cyc64) / t64 / 1e9,
            "other_coarse_operator": alt,
            "roofline": roof,
            "cycle_roofline": {
                "glups": value, "peak_gbs": hbm, "peak_source": src,
                "bytes_per_cell_cycle": _CYCLE_BYTES_MIXED,
                "achieved_gbs": value * _CYCLE_BYTES_MIXED, "frac": value * _CYCLE_BYTES_MIXED / hbm,
                "alg_min_bytes_per_cell_cycle": _CYCLE_BYTES_ALG_MIN,
                "achieved_gbs_alg_min": value * _CYCLE_BYTES_ALG_MIN,
                "frac_alg_min": value * _CYCLE_BYTES_ALG_MIN / hbm,
                "models": "78 B: FP32 V(2,2) with four smoother passes, residual+restriction and prolongation per "
                          "level plus one FP64 residual per cycle; 37.7 B: one fused down- and up-pass per level",
                **({"face_averaged_coarse_extra_bytes": _CYCLE_BYTES_FACES_EXTRA,
                    "frac_with_face_coarse_bytes": value * (_CYCLE_BYTES_MIXED + _CYCLE_BYTES_FACES_EXTRA) / hbm}
                   if coeff and args.coarse_coef == "faces" else {})},
            "setup_ms": {"mg_set_rhs": round(setup_ms, 3), "in_value": False},
            "alu_peaks_tflops": {"fp64_fma": alu[0], "fp32_fma": alu[1], "source": "mg_alu_peaks, measured this run"},
            "residual_f64_roofline": res_roof,
            "smoother_finest": _smoother_report(prof, cells),
            "kernel_families_ms": {k_: round(v[0], 3) for k_, v in prof.items() if v[1]},
            "kernel_families_launches": {k_: v[1] for k_, v in prof.items() if v[1]},
            "gpu_launches": launches,
            "e2e": {"value": cells * e2e_cycles / te2e / 1e9 * ws, "unit": UNIT,
                    "h2d_bytes_per_step": int(fh.numel() * 8 * (2 if coeff else 1)),
                    "d2h_bytes_per_step": int(uh.numel() * 8),
                    "includes": "mg_solve_host per step: H2D f,k (the k set-up overlaps the f copy) + set-up "
                                "(coefficient pyramid, coarsest inverse) + solve + D2H u"},
            "clocks": clocks,
        }
    F.close()
    del F64
    if rank == 0 and ws == 1 and not getattr(args, "no_other_configs", False):
        torch.cuda.empty_cache()
        out["other_configs"] = run_other_configs(dev, args.coarse_coef)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------------------
# the other configurations of the benchmark set, each timed with its own clock record (rank 0, N = 1)
# ------------------------------------------------------------------------------------------------------------
def _timed(fn, reps):
    """Mean seconds of reps calls of fn, CUDA events on the current stream around them (synchronised)."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = [fn() for _ in range(reps)]
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3 / reps


def _cfg_small(dev, cc):
    """2^3 roots of 16^3 (32,768 cells), -Laplace with the sin-product right-hand side, FP64 V(2,2), exactly 10
    cycles: launch-latency-bound, reported as microseconds per cycle."""
    import synthetic as syn
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest("uniform_2x16")
    f = syn.sin_product_rhs(R, n, keys).to(dev)
    F = Forest(R, n, keys, precision=0)
    F.set_rhs(f)
    u = torch.zeros_like(f)

    def run():
        u.zero_()
        return F.vcycle(u, 10)

    for _ in range(3):
        run()
    rels, t = _timed(run, 20)
    ue = syn.sin_product(R, n, keys).to(dev)
    err = float(torch.sqrt(((u - ue) ** 2).sum() / (R * n) ** 3))
    F.close()
    cells = len(keys) * n ** 3
    return {"workload": "uniform_2x16 (2^3 roots of 16^3, sin-product f)", "cells": cells, "dtype": "f64",
            "cycles": 10, "us_per_cycle": t / 10 * 1e6, "glups_per_cycle": cells * 10 / t / 1e9,
            "rel_residual_after_10": rels[-1], "l2_error_vs_exact": err,
            "timing": "20 repetitions of 10 cycles from u = 0 (each ends with the residual and the copy of u)"}


def _cfg_refined(dev, cc):
    """The refined 56 + 64 block forest of 32^3 blocks (3,932,160 cells), Gaussian bump plus noise, solved to
    1e-10 in FP64 (and with FP32 cycles inside FP64 defect correction for comparison)."""
    import synthetic as syn
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest("sphere_2x32")
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=1, device=dev)
    cells = len(keys) * n ** 3
    res = {"workload": "sphere_2x32 (56 + 64 blocks of 32^3, bump + noise f)", "cells": cells, "rtol": 1e-10}
    for name, prec, inner in (("fp64", 0, 1), ("fp32_in_fp64", 1, 4)):
        F = Forest(R, n, keys, precision=prec, inner_cycles=inner)
        F.set_rhs(f)
        u = torch.zeros_like(f)

        def run():
            u.zero_()
            return F.solve(u, rtol=1e-10, max_cycles=60)

        run()
        out, t = _timed(run, 5)
        cyc = out[-1][0]
        res[name] = {"time_to_rtol_ms": t * 1e3, "cycles": cyc, "glups_per_cycle": cells * cyc / t / 1e9,
                     "final_rel_residual": out[-1][1]}
        F.close()
    res["speedup_fp32_in_fp64"] = res["fp64"]["time_to_rtol_ms"] / res["fp32_in_fp64"]["time_to_rtol_ms"]
    return res


def _cfg_adjoint(dev, cc):
    """The differentiation workload: 4^3 roots of 32^3 refined twice around the sphere (448 + 512 blocks,
    31,457,280 cells), log-normal k, bump f; forward FP32-in-FP64 solve to 1e-10, then the adjoint solve (transposed
    V-cycles) giving dL/df and dL/dk for L = 1/2 ||u - u_t||^2."""
    import synthetic as syn
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest("sphere_4x32")
    k = syn.lognormal_k_rff(R, n, keys, seed=5, device=dev)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=6, device=dev)
    ut = syn.sin_target(R, n, keys, seed=7, device=dev)
    cells = len(keys) * n ** 3
    F = Forest(R, n, keys, coeff=True, precision=1, inner_cycles=4, coarse_coef=cc)
    t0 = time.perf_counter()
    F.set_rhs(f, k)
    torch.cuda.synchronize()
    first_setup_s = time.perf_counter() - t0
    u = torch.zeros_like(f)

    def fwd():
        u.zero_()
        return F.solve(u, rtol=1e-10, max_cycles=60)

    def adj():
        return F.adjoint(u, u - ut, want_k=True, rtol=1e-10)

    fwd()
    adj()
    fo, tf = _timed(fwd, 3)
    _ao, ta = _timed(adj, 3)
    _, ts = _timed(lambda: F.set_rhs(f, k), 3)
    F.close()
    return {"workload": "sphere_4x32 (448 + 512 blocks of 32^3, log-normal k, bump f, sin target)",
            "cells": cells, "coarse_coefficients": _COARSE_COEF_NAMES[cc], "forward_ms": tf * 1e3, "forward_cycles": fo[-1][0], "adjoint_ms": ta * 1e3,
            "forward_plus_adjoint_ms": (tf + ta) * 1e3, "setup_ms": ts * 1e3, "first_setup_s": first_setup_s,
            "forward_glups_per_cycle": cells * fo[-1][0] / tf / 1e9,
            "adjoint": "lambda = A^-T (u - u_t) to 1e-10 by defect correction with the transposed V-cycle, "
                       "dL/df = lambda, dL/dk face by face"}


def _cfg_batch(dev, cc):
    """256 independent single-root problems (block sizes 16..128, 0-2 refinement levels, log-normal k, U(-1, 1)
    f), each solved to 1e-8 with FP32 cycles inside FP64 defect correction, one graph launch per step."""
    import synthetic as syn
    from paper_2403_08063_gb300 import Batch
    t0 = time.perf_counter()
    problems = syn.batch_problems(count=256, seed=0)
    leaves, ns = syn.batch_leaves(problems)
    f, k = syn.batch_fields(problems, seed=0, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    cells = f.numel()
    t0 = time.perf_counter()
    B = Batch(leaves, ns, coeff=True, inner_cycles=5, coarse_coef=cc)
    B.set_rhs(f, k)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    u = torch.zeros_like(f)

    def run():
        u.zero_()
        return B.solve(u, rtol=1e-8, max_cycles=60)

    run()
    out, t = _timed(run, 2)
    cyc = max(out[-1][0])
    info = B.info()
    mode, tails = B.tail_mode(), B.tail_levels()
    B.close()
    del f, k, u
    torch.cuda.empty_cache()
    return {"workload": "batch_256", "problems": 256, "cells": cells, "groups": info["groups"], "rtol": 1e-8,
            "coarse_coefficients": _COARSE_COEF_NAMES[cc], "tail_mode": mode, "persistent_tail_from_level": tails,
            "solve_ms": t * 1e3, "cycles_max": cyc, "glups_per_cycle": cells * cyc / t / 1e9,
            "worst_rel_residual": max(out[-1][1]), "inputs_s": gen_s, "create_and_first_setup_s": setup_s,
            "timing": "2 solves after 1 warm-up, graph-launched"}


def run_other_configs(dev, cc):
    out = {}
    for name, fn in (("c1_uniform_2x16_fp64", _cfg_small), ("c2_sphere_2x32", _cfg_refined),
                     ("c5_sphere_4x32_adjoint", _cfg_adjoint), ("c4_batch_256", _cfg_batch)):
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        w0 = time.perf_counter()
        try:
            rec = fn(dev, cc)
        except Exception as e:  # a failing extra configuration must not hide the headline line
            rec = {"error": f"{type(e).__name__}: {e}"}
        rec["wall_s"] = time.perf_counter() - w0
        rec["clocks"] = sampler.stop()
        out[name] = rec
        torch.cuda.empty_cache()
    return out


def run_batch(args):
    """Batched workload: independent problems with block sizes 16^3..128^3, each solved to 1e-8."""
    import synthetic as syn
    from paper_2403_08063_gb300 import Batch
    dist, rank, ws, local = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    count = 256 if args.workload == "batch_256" else 32
    problems = syn.batch_problems(count=count, seed=0)
    leaves, ns = syn.batch_leaves(problems)
    f, k = syn.batch_fields(problems, seed=0, device=dev)
    cells = f.numel()
    B = Batch(leaves, ns, coeff=True, inner_cycles=args.inner_cycles, coarse_coef=args.coarse_coef)
    B.set_rhs(f, k)
    if args.tail == "-1":
        B.set_tail_off()
    u = torch.zeros_like(f)
    rtol = 1e-8

    def step():
        u.zero_()
        return B.solve(u, rtol=rtol, max_cycles=60)

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    _barrier(dist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    runs = []
    for _ in range(args.steps):
        runs.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    clocks = sampler.stop()
    t = _max_over_ranks(dist, e0.elapsed_time(e1) / 1e3)
    cyc_run = [max(c) for c, _ in runs]
    value = cells * sum(cyc_run) / t / 1e9 * ws
    # kernel families from one profiled solve (graphs off while profiling)
    B.profile(True)
    torch.cuda.nvtx.range_push("mg_batch_profiled")
    step()
    torch.cuda.nvtx.range_pop()
    prof = B.profile_read()
    B.profile(False)
    if rank == 0:
        out = {
            "metric": "GLUPS per V(2,2) cycle (batched FP32-in-FP64 solves to 1e-8)", "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 cycles + f64 outer",
            "data": "synthetic",
            "config": {"workload": args.workload, "problems": count, "cells": cells, "groups": B.info()["groups"],
                       "rtol": rtol, "inner_cycles": args.inner_cycles,
                       "coarse_coefficients": _COARSE_COEF_NAMES[args.coarse_coef],
                       "persistent_tail_from_level": B.tail_levels(),
                       "tail_mode": {0: "every level launched", 1: "each group's own persistent tail",
                                     2: "one joint persistent tail per V-cycle"}[B.tail_mode()],
                       "graphs": "one defect-correction step of "
                       "all groups per graph launch", "l2": "inputs larger than L2 (no flush)"},
            "cycles_per_solve_max": cyc_run, "cycles_per_problem_last": runs[-1][0],
            "worst_rel_residual": max(runs[-1][1]),
            "kernel_families_ms_profiled_solve": {k_: round(v[0], 3) for k_, v in prof.items() if v[1]},
            "gpu_launches_profiled_solve": sum(v[1] for v in prof.values()),
            "clocks": clocks,
        }
        print(json.dumps(out), flush=True)
    B.close()
    if dist is not None:
        dist.destroy_process_group()


def _sync_time(fn):
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def run_paper_bench(args):
    """The paper's benchmark workload (Sec. 6) on one GPU: R^3 roots refined once, a quarter of them once more
    (22 R^3 blocks of 64^3, R = 4), V(3,3) damped-Jacobi cycles with 256 coarsest Jacobi sweeps, ghost-only
    interfaces, FP64.  A step is 20 cycles (the paper times 100).  Reports t_cycle, GLUPS per cycle, the finest-level
    Jacobi sweep against the paper's 24 B/LUP light-speed model at this GPU's measured bandwidth, and the coarsest
    solver's share of the cycle (paper: 1.64-5.15 % with generated communication)."""
    import synthetic as syn
    from paper_2403_08063_gb300 import Forest
    dev = torch.device("cuda", 0)
    R, n = 4, 64
    keys = syn.paper_benchmark_forest(R)
    cells = len(keys) * n ** 3
    f = syn.uniform_rhs(len(keys), n, seed=0).to(dev)
    F = Forest(R, n, keys, interface_flux=False, precision=0, nu1=3, nu2=3, smoother="jacobi", omega=0.8,
               coarse_iters=256)
    F.set_rhs(f)
    u = torch.zeros_like(f)
    per_step = 20
    for _ in range(args.warmup):
        F.vcycle(u, per_step)
    sampler = ClockSampler(0)
    sampler.start()
    _, t = _sync_time(lambda: [F.vcycle(u, per_step) for _ in range(args.steps)])
    F.profile(True)
    F.vcycle(u, per_step)
    torch.cuda.synchronize()
    prof = F.profile_read()
    F.profile(False)
    clocks = sampler.stop()
    ncyc = per_step * args.steps
    tcyc = t / ncyc
    fin = prof.get("smooth_f64_finest", (0.0, 0))
    sweep_s = fin[0] / 1e3 / max(1, fin[1])
    hbm, src = _peaks()
    prof_total = sum(v[0] for v in prof.values())
    print(json.dumps({
        "metric": "t_cycle of V(3,3) damped-Jacobi cycles, the paper's benchmark workload (FP64)",
        "value": tcyc * 1e3, "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "paper_bench", "roots": R, "blocks": len(keys), "block": f"{n}^3", "cells": cells,
                   "levels": F.levels(), "cycle": "V(3,3) damped Jacobi (omega 0.8), 256 coarsest Jacobi sweeps",
                   "cycles_timed": ncyc, "interfaces": "ghost-only (paper)"},
        "glups_per_cycle": cells / tcyc / 1e9,
        "finest_jacobi_sweep": {"ms": sweep_s * 1e3, "glups": cells / sweep_s / 1e9,
                                "light_speed_model_glups": hbm * 1e9 / 24.0 / 1e9,
                                "frac_of_model": cells / sweep_s / (hbm * 1e9 / 24.0), "peak_source": src,
                                "model": "24 B per LUP (the paper's Sec. 6 model: u load + store, f load, FP64)"},
        "coarse_solve_fraction": prof.get("coarse_f64", (0.0, 0))[0] / prof_total if prof_total else None,
        "kernel_families_ms_per_20_cycles": {k_: round(v[0], 3) for k_, v in prof.items() if v[1]},
        "clocks": clocks,
    }), flush=True)


def _vw_error(R, n, keys, u, g, dev, chunk_cells=1 << 26):
    """Volume-weighted L2 error sqrt(sum h^3 (u - g)^2) of u (n_leaves, n^3) against g at the cell centres, evaluated
    a few leaves at a time, so that the centre coordinates never exist for the whole forest at once."""
    import synthetic as syn
    per = max(1, chunk_cells // n ** 3)
    acc = 0.0
    for s in range(0, len(keys), per):
        sl = slice(s, min(s + per, len(keys)))
        c = syn.cell_centres(R, n, keys, device=dev, leaf_slice=sl).reshape(sl.stop - sl.start, -1, 3)
        exact = torch.sin(np.pi * c[..., 0]) * torch.sin(np.pi * c[..., 1]) * torch.sinh(np.sqrt(2) * np.pi * c[..., 2])
        h3 = torch.tensor([(1.0 / (R * 2 ** k[0] * n)) ** 3 for k in keys[sl]], dtype=torch.float64, device=dev)
        acc += float((h3[:, None] * (u[sl] - exact) ** 2).sum())
        del c, exact
    return math.sqrt(acc)


def run_paper_table(args):
    """Table err_analysis (Sec. 5) on the GPU: -Laplace u = 0 with Dirichlet data u = sin(pi x) sin(pi y)
    sinh(sqrt(2) pi z) on the 56 + 64 block geometry, the paper's V(3,3) damped-Jacobi cycle with 256 coarsest
    sweeps and ghost-only interfaces, FP64, solved to a 1e-13 relative residual; L2 (volume-weighted) error against
    the exact solution for the block sizes in --table-sizes (16 .. 256) and the three coarse-to-fine variants, with
    the paper's values.  The 256^3 row (2.0e9 cells) holds about 130 GB on the device; its error is evaluated a few
    leaves at a time."""
    import synthetic as syn
    from paper_2403_08063_gb300 import Forest
    dev = torch.device("cuda", 0)
    R, _, keys = syn.workload_forest("sphere_2x4")
    paper = {16: (0.235, 1.067e-2, 3.017e-3), 32: (0.227, 5.255e-3, 7.215e-4), 64: (0.224, 2.611e-3, 1.764e-4),
             128: (0.222, 1.302e-3, 4.361e-5), 256: (0.221, 6.499e-4, 1.084e-5)}
    g = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sinh(np.sqrt(2) * np.pi * z)  # noqa: E731
    sizes = [int(v) for v in args.table_sizes.split(",")]
    rows = {}
    sampler = ClockSampler(0)
    sampler.start()
    for n in sizes:
        for variant in (0, 1, 2):  # second order (the paper's scheme), first order, constant
            F = Forest(R, n, keys, interface_flux=False, precision=0, nu1=3, nu2=3, smoother="jacobi", omega=0.8,
                       coarse_iters=256, c2f_variant=variant)
            f = torch.zeros((len(keys), n ** 3), dtype=torch.float64, device=dev)
            F.set_rhs(f)
            F.set_boundary(syn.boundary_values(R, n, keys, g, device=dev))
            u = f  # f is zero and no longer needed after set_rhs: the solve starts from it
            (cyc, rel), ts = _sync_time(lambda: F.solve(u, rtol=1e-13, max_cycles=80, raise_on_failure=False))
            F.close()
            del F
            torch.cuda.empty_cache()
            err = _vw_error(R, n, keys, u, g, dev)
            rows.setdefault(n, {})[("second", "first", "constant")[variant]] = {
                "error": err, "paper": paper[n][2 - variant], "ratio": err / paper[n][2 - variant], "cycles": cyc,
                "rel_residual": rel, "solve_s": ts, "cells": len(keys) * n ** 3}
            del u, f
            torch.cuda.empty_cache()
    clocks = sampler.stop()
    ns = sorted(rows)
    kappa = {o: [rows[ns[i + 1]][o]["error"] / rows[ns[i]][o]["error"] for i in range(len(ns) - 1)]
             for o in ("second", "first", "constant")}
    print(json.dumps({"metric": "L2 error of Table err_analysis (paper's accuracy problem)", "unit": "L2 error",
                      "workload": "paper_table", "rows": {str(k): v for k, v in rows.items()}, "kappa": kappa,
                      "paper_kappa": {"second": [0.239, 0.244, 0.247, 0.249], "first": [0.493, 0.497, 0.499, 0.499],
                                      "constant": [0.966, 0.984, 0.992, 0.996]}, "clocks": clocks}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="uniform_8x64_k")
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--inner-cycles", type=int, default=0,
                    help="FP32 V-cycles per FP64 defect-correction step (0: 5 for the batches solved to 1e-8 and "
                         "for variable-k solves with face-averaged coarse levels, else 4)")
    ap.add_argument("--tail", default="auto",
                    help="level from which the persistent tail kernel runs the FP32 V-cycle (-1: off; auto: tuned)")
    ap.add_argument("--smoother-shape", default="",
                    help="FP32 smoother launch shape of the finest level, e.g. 2,16,16,2,4 (default: tuned)")
    ap.add_argument("--coarse-coef", choices=sorted(_COARSE_COEF_NAMES), default="faces",
                    help="coarse-level coefficients with variable k: faces (each coarse face the mean of the finer "
                         "faces it covers) or k (rediscretised from the mean of the children's k)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the other configurations (small FP64 forest, refined forest, adjoint, batch)")
    ap.add_argument("--table-sizes", default="16,32,64,128",
                    help="block sizes of the paper_table workload (256 needs about 130 GB on the device)")
    args = ap.parse_args()
    if args.inner_cycles <= 0:
        # the fastest counts measured on a GB300: 5 for the batches (to 1e-8) and for variable-k solves with
        # face-averaged coarse levels (10 cycles to 1e-10 at 512^3, against 12 with 4 or 6), else 4
        faces_k = args.coarse_coef == "faces" and WORKLOADS[args.workload][1]
        args.inner_cycles = 5 if args.workload.startswith("batch") or faces_k else 4
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("batch"):
        run_batch(args)
    elif args.workload == "paper_bench":
        run_paper_bench(args)
    elif args.workload == "paper_table":
        run_paper_table(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
