#!/usr/bin/env python
"""Benchmark of the implicit JFNK step on GB300.

A step is one Crank-Nicolson implicit time step (Newton + preconditioned
GMRES + Jacobian-free products) of the 2-D Kelvin-Helmholtz workload on a
512 x 512 periodic grid at CFL 10, Newton tolerance 1e-8 (seeded synthetic
initial condition, see paper_1610_10053_gb300.inputs).  The headline value
is the mixed-precision path (FP64 residual and differencing, FP32 Krylov
basis and preconditioner) in cell-steps/s; the plain FP64 GPU path is timed
in the same run.  Multi-GPU runs are independent replicas (weak scaling, no
collective on the data path).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl music|reference]
"""
from __future__ import annotations

import argparse
import contextlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-steps/s at Newton tol 1e-8, mixed vs FP64; residual HBM GB/s; p99 step ms"
L2_FLUSH_BYTES = 512 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, ws: int, device) -> float:
    """The largest of the ranks' values (a replica job takes its slowest
    rank's time)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, cells: int, steps: int, total_ms: float) -> float:
    """Whole-job cell-steps/s: the cell-steps of all ranks over the slowest
    rank's time (replicas: every rank advances its own grid)."""
    return ws * cells * steps / (total_ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOADS = {
    "kh512": ("Kelvin-Helmholtz 2-D, 512x512 periodic, CFL 10, Newton tol 1e-8, GMRES(30)",
              lambda I, r: I.kelvin_helmholtz(n=512, seed=2 + r)),
    "kh2048": ("Kelvin-Helmholtz 2-D, 2048x2048 periodic, CFL 10, Newton tol 1e-8, GMRES(30)",
               lambda I, r: I.kelvin_helmholtz(n=2048, seed=2 + r)),
    "rt64x192": ("Rayleigh-Taylor 2-D, 64x192, CFL 5, Newton tol 1e-8, GMRES(30)",
                 lambda I, r: I.rayleigh_taylor()),
    "rt64x192_scalars": ("Rayleigh-Taylor 2-D, 64x192, two passive scalars (unpreconditioned scalar JFNK), "
                         "CFL 5, Newton tol 1e-8, GMRES(30)",
                         lambda I, r: I.rayleigh_taylor(scalars=True)),
    "rt_paper": ("Rayleigh-Taylor 2-D at the paper's settings: 100x300, CFL_hydro 0.8, unpreconditioned JFNK, "
                 "two passive scalars, Newton tol 1e-8, GMRES(30)",
                 lambda I, r: I.rt_paper()),
    "tgv128": ("Taylor-Green vortex 3-D, 128^3 periodic, CFL 20, Newton tol 1e-8, GMRES(30)",
               lambda I, r: I.taylor_green(n=128)),
    "tgv256": ("Taylor-Green vortex 3-D, 256^3 periodic, CFL 20, Newton tol 1e-8, GMRES(30)",
               lambda I, r: I.taylor_green(n=256)),
    "wedge256": ("2-D spherical wedge 256 (r) x 128 (theta), radiative diffusion, polytrope n=3 background, "
                 "dt = 100x acoustic CFL, Newton tol 1e-8, GMRES(30)",
                 lambda I, r: I.spherical_wedge(seed=5 + r)),
}


def workload(name: str, rank: int):
    from paper_1610_10053_gb300 import inputs as I
    return WORKLOADS[name][1](I, rank)


# the oracle's sample for workloads too large to time a full step of on the
# host within a minute: the same setup on a smaller grid (cell-steps/s is a rate)
CPU_SAMPLES = {"tgv128": ("TGV 64^3 (the same setup on 1/8 of the cells)", lambda I: I.taylor_green(n=64)),
               "tgv256": ("TGV 64^3 (the same setup on 1/64 of the cells)", lambda I: I.taylor_green(n=64)),
               "kh2048": ("KH 512^2 (the same setup on 1/16 of the cells)", lambda I: I.kelvin_helmholtz(n=512))}


def time_steps(grid, steps, stream, flush):
    """Per-step device times (ms) with CUDA events on the launching stream,
    L2 flushed between steps outside the events."""
    import torch
    times, stats = [], []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = grid.step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(st)
    return times, stats


def run_music(args):
    import torch
    import torch.distributed as dist
    from paper_1610_10053_gb300 import binding as B

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    prob = workload(args.workload, rank)
    N = prob.ncells
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # CPU baseline first (rank 0, N = 1 only), so it never overlaps GPU timing
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        if args.workload in CPU_SAMPLES:
            from paper_1610_10053_gb300 import inputs as I
            label, make = CPU_SAMPLES[args.workload]
            cpu = cpu_baseline(make(I), label)
        else:
            cpu = cpu_baseline(prob, args.workload)

    # the FP64 / FP32 ceilings of this GPU, measured in this run (the residual
    # stencil is FP64-bound; the roofline is reported against these)
    alu_peaks = B.measure_peaks()
    result = {}
    for name, prec in (("mixed", B.MIXED), ("fp64", B.FP64)):
        if name == "fp64" and args.skip_fp64:
            continue
        g = B.Grid(prob, precision=prec)
        g.set_state(prob.U)
        if prob.q is not None:
            g.set_scalars(prob.q)
        tune = g.autotune()  # tile shapes and preconditioner stages (untimed)
        for _ in range(args.warmup):
            g.step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = B.kernel_launches()
        with ClockSampler(local) as clk:
            times, stats = time_steps(g, args.steps, stream, flush)
        launches = B.kernel_launches() - l0
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        # the Jv stencil's launch time: CUDA events around every launch of a
        # pass of the same number of steps right after the timed region (the
        # recorded solver graph admits no events, so this pass is
        # host-sequenced; the kernels are the same)
        g.profile(True)
        time_steps(g, args.steps, stream, flush)
        prof = {k: g.profile_read(c) for k, c in (("jv", B.PROF_JV), ("precond", B.PROF_PRECOND),
                                                   ("residual", B.PROF_RESIDUAL), ("vector", B.PROF_VECTOR))}
        g.profile(False)
        jv_form = ("diff" if g.jv_form() == B.JV_DIFF32 else "fd") if prec == B.MIXED else "fd"
        total_ms = max_over_ranks(float(np.sum(times)), ws, "cuda")
        result[name] = dict(total_ms=total_ms, times=times, stats=stats, launches=launches,
                            clocks=clk.summary(), grid=g, prof=prof, jv_form=jv_form,
                            tiles={"stencil": list(tune["stencil_tile"]), "residual": list(tune["residual_tile"]),
                                   "precond": list(tune["precond_tile"]),
                                   "precond_stages": tune["precond_stages"]} if tune["tunable"] else None)
    mixed = result["mixed"]
    value = job_rate(ws, N, args.steps, mixed["total_ms"])
    fp64_value = None
    if "fp64" in result:
        fp64_value = job_rate(ws, N, args.steps, result["fp64"]["total_ms"])

    mixed["kernels"] = kernel_classes(mixed, prob)
    roof = roofline(mixed, prob, mixed["jv_form"], alu_peaks)
    final_diag = mixed["grid"].diagnostics()
    if prob.q is not None:
        final_diag["scalar_mixing_width"] = mixed["grid"].scalar_mixing_width()
    e2e = end_to_end(mixed["grid"], prob, stream, max(2, min(args.steps, 5)))
    for r in result.values():
        r["grid"].close()
    series = None
    if args.series > 0 and rank == 0:
        series = run_series(prob, args.series, max(1, args.every))
    dt_study = None
    if args.dt_study > 0 and rank == 0:
        dt_study = run_dt_study(args.dt_study, args.dt_study_t)
    convergence = None
    if args.convergence > 0 and rank == 0:
        convergence = run_convergence(args.convergence, args.conv_t)
    serving = None
    if not args.no_serving and ws == 1:
        serving = run_serving(args.serve_solves, lane_cells=args.serve_lane_cells)
        # a mix of small grids only, which cannot fill the GPU one solve at a time
        serving = {"mix": serving, "small_grids": run_serving(
            args.serve_solves, lane_cells=args.serve_lane_cells, grids=((64, 64), (128, 128)), label="small"),
            "burst_64": run_burst(args.serve_solves, lane_cells=args.serve_lane_cells)}

    if rank != 0:
        return
    t = np.array(mixed["times"])
    st = mixed["stats"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "cell-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": float(t.mean()),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 residual + f32 Krylov (mixed)",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0],
                   "cells": N, "precision": "mixed", "l2": "flushed (512 MiB write) between timed steps",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "solver": "recorded CUDA graph per Newton attempt",
                   "tiles": {k: r["tiles"] for k, r in result.items()}},
        "fp64_value": fp64_value,
        "mixed_over_fp64": (value / fp64_value) if fp64_value else None,
        "step_ms_p50": float(np.percentile(t, 50)),
        "step_ms_p99": float(np.percentile(t, 99)),
        "newton_its_per_step": float(np.mean([s["newton_its"] for s in st])),
        "gmres_its_per_step": float(np.mean([s["gmres_its"] for s in st])),
        "scalar_gmres_its_per_step": float(np.mean([s["scalar_gmres_its"] for s in st])) if prob.q is not None
        else None,
        "fp64_ms_per_step": float(np.mean(result["fp64"]["times"])) if "fp64" in result else None,
        "roofline": roof,
        "kernels": mixed["kernels"],
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clocks"],
        "serving": serving,
        "series": series,
        "dt_study": dt_study,
        "convergence": convergence,
        "final_diagnostics": final_diag,
        "sim_time": float(sum(x["dt"] for x in mixed["stats"])),
    }
    print(json.dumps(line))


# Roofline models of the step's three kernel classes on the fused 2-D grids
# (per cell; every +, -, *, / counts 1 and an FMA 2; bytes are the
# algorithmic reads and writes of one launch).
#
# Jacobian-free product, FP64 form: forming U + eps v 8, e and p 2, two face
# velocities 6, eight van Leer slopes 48, mass and energy fluxes 12, momentum
# fluxes 20, residual assembly 43, Jv = v - c (R - R_U) 12.
JV_FD_FLOPS_PER_CELL_2D = 151
JV_FD_BYTES_PER_CELL_2D = 96      # U (4 x 8), R(U) (4 x 8), v (4 x 4) read, Jv (4 x 4) written
# Jacobian-free product, difference form (FP32): the differences of e, u, v
# by the quotient rule 16, eight limited slopes with their differences 144,
# upwind mass and energy fluxes 32, four momentum fluxes 44, residual
# differences and Jv = v - dt/2 dR 45.
JV_DIFF_FLOPS_PER_CELL_2D = 281
JV_DIFF_BYTES_PER_CELL_2D = 80    # v (16), the 12 linearisation planes (48) read, Jv (16) written
# ncu dram__bytes_read.sum + dram__bytes_write.sum per cell of one launch on
# KH 2048^2 (state above L2 size), scaled to the bench's cells; None where
# the kernel changed after its last 2048^2 capture
JV_DIFF_TRAFFIC_B_PER_CELL_2D = None
JV_FD_TRAFFIC_B_PER_CELL_2D = None
# Preconditioner application (FP32), K Jacobi sweeps: right-hand side 12,
# each sweep 15, back substitution 33.
def precond_flops_per_cell(K):
    return 12 + 15 * K + 33
PRECOND_BYTES_PER_CELL_2D = 52    # r (16), coefficients a_x, a_y, gamma p, gamma E, D (20) read, z (16) written
PRECOND_TRAFFIC_B_PER_CELL_2D = None  # (changed since its 2048^2 capture)
# Residual-type evaluation (FP64): R(U) as in the product without U + eps v,
# and the assembly sign ((U - C^n) - dt/2 R) 12.
RES_FLOPS_PER_CELL_2D = 143
RES_BYTES_PER_CELL_2D = 176       # U, C^n read, F and R(U) written (4 x 8 each), linearisation planes (48)
RES_TRAFFIC_B_PER_CELL_2D = 166.4 # ncu, F mode on KH 2048^2, 16 x 16 tile
# ncu dram bytes of one launch of each kernel on the bench's own KH 512^2
# workload with its tuned tiles (MUSIC_TILES=32x16,16x16,32x32,3), cold L2:
# the launch's reads; its writes stay in the 126 MB L2 (profiles/*_kh512.md).
# None: the kernel changed since its last capture of DRAM bytes.
TRAFFIC_KH512 = {"residual": 17.626e6, "jv": 16.88e6, "precond": None}
# Peaks derived from the part's unit counts and clock (152 SMs, 2.07 GHz):
# FP64 2 FMA per SM per clock; FP32 128 FMA per SM per clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def kernel_classes(mixed, prob):
    """Live per-launch times of the three profiled classes (CUDA events
    around every launch, on its stream, in a pass of the timed number of
    steps right after the timed region) and their share of the step."""
    out = {}
    step_ms = mixed["total_ms"] / max(1, len(mixed["times"]))
    for name, (n, ms) in mixed["prof"].items():
        if n:
            out[name] = {"launches": n, "ms_per_launch": ms / n, "ms_per_step": ms / len(mixed["times"]),
                         "share_of_step": ms / len(mixed["times"]) / step_ms}
    # what no class covers: the recorded graph's control kernels and the gaps
    # between dependent launches
    rest = step_ms - sum(v["ms_per_step"] for v in out.values())
    out["unattributed"] = {"ms_per_step": rest, "share_of_step": rest / step_ms}
    return out


def roofline(mixed, prob, jv_form, alu=None):
    """The roofline of the class that takes the most device time per step,
    against the FP64 or FP32 FMA throughput measured in this run
    (music_measure_peaks; the unit-count figure when none was measured)."""
    # many small kernels in "vector", none in "unattributed": no one roofline for either
    ks = {k: v for k, v in mixed["kernels"].items() if k not in ("vector", "unattributed")}
    if not ks:
        return None
    name = max(ks, key=lambda k: ks[k]["ms_per_step"])
    per = ks[name]["ms_per_launch"]
    N = prob.ncells
    fused = prob.nd == 2 and prob.geometry == 0 and not prob.conduct
    hbm, src = peaks()
    if name == "jv" and jv_form == "diff" and fused:
        flops, peak, unit, bpc, tpc = (JV_DIFF_FLOPS_PER_CELL_2D, FP32_PEAK_TFLOPS, "FP32",
                                       JV_DIFF_BYTES_PER_CELL_2D, JV_DIFF_TRAFFIC_B_PER_CELL_2D)
        kern = "k_jvdiff2d (Jacobian-free product, difference form)"
    elif name == "jv":
        flops, peak, unit, bpc, tpc = (JV_FD_FLOPS_PER_CELL_2D, FP64_PEAK_TFLOPS, "FP64",
                                       JV_FD_BYTES_PER_CELL_2D, JV_FD_TRAFFIC_B_PER_CELL_2D)
        kern = "k_fused2d (Jacobian-free product mode)" if fused else "multi-pass stencil (Jacobian-free product mode)"
    elif name == "precond":
        flops, peak, unit, bpc, tpc = (precond_flops_per_cell(prob.sweeps), FP32_PEAK_TFLOPS, "FP32",
                                       PRECOND_BYTES_PER_CELL_2D, PRECOND_TRAFFIC_B_PER_CELL_2D)
        kern = "k_precond_fused2d (preconditioner application, all stages)"
    else:
        flops, peak, unit, bpc, tpc = (RES_FLOPS_PER_CELL_2D, FP64_PEAK_TFLOPS, "FP64", RES_BYTES_PER_CELL_2D,
                                       RES_TRAFFIC_B_PER_CELL_2D)
        kern = "k_fused2d (R / C^n / F modes)"
    if not fused:
        return {"kernel": kern, "bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "launches": ks[name]["launches"], "ms_per_launch": per,
                "note": "per-cell model given for the fused 2-D kernels only"}
    derived = peak
    if alu:
        peak = alu["fp64_fma_tflops"] if unit == "FP64" else alu["fp32_fma_tflops"]
    achieved = flops * N / (per / 1e3) / 1e12
    if N == 512 * 512 and (name != "jv" or jv_form == "diff"):
        traffic = TRAFFIC_KH512[name]
        tnote = ("ncu dram read+write of one launch of this workload (tuned tiles, cold L2)" if traffic is not None
                 else "kernel changed since its last ncu capture of DRAM bytes")
    else:
        traffic = tpc * N if tpc else None
        tnote = ("ncu dram read+write per cell on KH 2048^2, scaled to this launch's cells" if tpc
                 else "kernel changed since its last ncu capture of DRAM bytes")
    return {"kernel": kern, "class": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_note": tnote,
            "launches": ks[name]["launches"], "ms_per_launch": per, "flops_per_cell": flops,
            "timing": "CUDA events around each launch, same-length pass after the timed region",
            "peak_note": ("%s FMA throughput measured in this run by music_measure_peaks (unit-count figure "
                          "152 SM x %s x 2.07 GHz = %.3f)" % (unit, "2 DFMA/clk" if unit == "FP64" else "128 FFMA/clk",
                                                             derived)) if alu else
                         ("%s peak derived from unit counts and clock (152 SM x %s x 2.07 GHz)"
                          % (unit, "2 DFMA/clk" if unit == "FP64" else "128 FFMA/clk")),
            "measured_alu_peaks": alu,
            "hbm_view": {"achieved_gbs": bpc * N / (per / 1e3) / 1e9, "peak_gbs": hbm, "peak_source": src,
                         "bytes_per_cell": bpc, "frac": bpc * N / (per / 1e3) / 1e9 / hbm if hbm else None}}


def end_to_end(grid, prob, stream, steps):
    """Same metric through the public API with host buffers: every step copies
    the state host -> device (pinned), steps, and copies it back."""
    import torch
    n = grid.n
    host_in = torch.from_numpy(prob.U.copy()).pin_memory()
    host_out = torch.empty(n, dtype=torch.float64).pin_memory()
    grid.set_state(host_in)
    grid.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        grid.set_state(host_in)
        grid.step()
        grid.get_state_into(host_out)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return {"value": prob.ncells * steps / el, "unit": "cell-steps/s", "h2d_bytes_per_step": n * 8,
            "d2h_bytes_per_step": n * 8, "steps": steps}


def serving_mix(nsolves=256, seed=4, grids=((64, 64), (128, 128), (256, 512), (512, 512))):
    """The serving workload: a seeded Poisson stream of solves drawn from the
    2-D Rayleigh-Taylor and Kelvin-Helmholtz setups, grids uniform over
    `grids` ({64^2, 128^2, 256x512, 512^2} by default), 20 implicit steps
    each."""
    from paper_1610_10053_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nsolves):
        nx, ny = grids[int(rng.integers(len(grids)))]
        if rng.integers(2) == 0:
            p = I.rayleigh_taylor(nx=nx, ny=ny, nsteps=20)
        else:
            p = I.kelvin_helmholtz(n=nx, ny=ny, seed=100 + i, nsteps=20)
        out.append(p)
    gaps = rng.exponential(1.0, size=nsolves)
    return out, gaps


def serve(probs, gaps, max_active, lane_cells):
    """One pass of the mix through the solve server (mixed precision, autotune
    on): arrivals at the given gaps, every result waited for."""
    from paper_1610_10053_gb300 import binding as B
    tickets = []
    with B.Server(max_active=max_active, batch_max_cells=lane_cells, autotune=True) as srv:
        start = time.perf_counter()
        t = start
        for p, gp in zip(probs, gaps):
            t += gp
            d = t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit(p, B.MIXED))
        res = [srv.wait(tk) for tk in tickets]
        wall = time.perf_counter() - start
        lat = srv.step_times()
        st = srv.stats()
    req = [r["total_ms"] for r in res]
    return {"completed": sum(r["status"] == 0 for r in res), "wall_s": wall,
            "batch_lane_max_cells": lane_cells,
            "batch_lane_solves": sum(1 for p in probs if 0 < lane_cells and p.ncells <= lane_cells),
            "cell_steps_per_s": st["cell_steps"] / wall,
            "step_ms_p50": float(np.percentile(lat, 50)), "step_ms_p99": float(np.percentile(lat, 99)),
            "request_ms_p50": float(np.percentile(req, 50)), "request_ms_p99": float(np.percentile(req, 99)),
            "queue_ms_p50": float(np.percentile([r["queue_ms"] for r in res], 50)),
            "queue_ms_p99": float(np.percentile([r["queue_ms"] for r in res], 99))}


def run_serving(nsolves=256, max_active=16, lane_cells=16384,
                grids=((64, 64), (128, 128), (256, 512), (512, 512)), label="mix"):
    """Continuous batching through the solve server (mixed precision), with
    the batch lane off and on (solves of at most `lane_cells` cells advance
    together in one launch per round), against the same solves run one after
    another on the plain FP64 GPU path (all of them)."""
    from paper_1610_10053_gb300 import binding as B
    probs, gaps = serving_mix(nsolves, grids=grids)
    cells = sum(p.ncells * p.nsteps for p in probs)
    t0 = time.perf_counter()
    for p in probs:
        with B.Grid(p, precision=B.FP64) as g:
            g.set_state(p.U)
            g.run()
    seq_s = time.perf_counter() - t0
    seq_rate = cells / seq_s
    # arrivals: mean gap chosen so that about `max_active` solves overlap on
    # the sequential service time
    gaps = gaps * (seq_s / nsolves / max_active)
    out = {"mix": label, "solves": nsolves, "grids": ["%dx%d" % g for g in grids], "max_active": max_active,
           "autotune": True, "cell_steps": cells, "sequential_fp64_cell_steps_per_s": seq_rate,
           "sequential_fp64_solves": nsolves, "mean_gap_ms": 1e3 * float(np.mean(gaps))}
    for name, lc in (("lane_off", 0), ("lane_on", lane_cells)):
        r = serve(probs, gaps, max_active, lc)
        r["over_sequential_fp64"] = r["cell_steps_per_s"] / seq_rate
        out[name] = r
    # request latency below saturation: the same solves arriving at 70 % of
    # the throughput the server reached (lane off) above
    load = 0.7
    gap70 = cells / len(probs) / (load * out["lane_off"]["cell_steps_per_s"])
    r = serve(probs, np.asarray(gaps) / np.mean(gaps) * gap70, max_active, 0)
    r["offered_load"] = load
    r["mean_gap_ms"] = 1e3 * gap70
    out["lane_off_70pct_load"] = r
    # the headline row: the better of the two
    best = max(("lane_off", "lane_on"), key=lambda k: out[k]["cell_steps_per_s"])
    out["best"] = best
    for k in ("cell_steps_per_s", "step_ms_p50", "step_ms_p99", "request_ms_p50", "request_ms_p99",
              "queue_ms_p99", "over_sequential_fp64", "completed"):
        out[k] = out[best][k]
    return out


def run_burst(nsolves=256, max_active=16, lane_cells=16384):
    """A burst of small solves: the mix's 64^2 setups only, all arriving at
    once, through the server with the batch lane off (max_active solves on
    the GPU at a time, each on the whole GPU) and on (every resident solve
    one CTA of one batched launch per round)."""
    probs, gaps = serving_mix(nsolves, grids=((64, 64),))
    zero = np.zeros_like(np.asarray(gaps))
    out = {"mix": "burst of 64x64 solves, all arriving at once", "solves": nsolves, "max_active": max_active,
           "cell_steps": sum(p.ncells * p.nsteps for p in probs)}
    for name, lc in (("lane_off", 0), ("lane_on", lane_cells)):
        out[name] = serve(probs, zero, max_active, lc)
    out["best"] = max(("lane_off", "lane_on"), key=lambda k: out[k]["cell_steps_per_s"])
    out["lane_on_over_lane_off"] = out["lane_on"]["cell_steps_per_s"] / out["lane_off"]["cell_steps_per_s"]
    return out


def run_series(prob, nsteps, every):
    """Diagnostics over a run (mixed precision, after the timed part): the
    density-based mixing width of Sec. 3 and, with scalars, the scalar-based
    one, and the maximum speed (the velocity residual of Sec. 6's hydrostatic
    test), every `every` steps."""
    from paper_1610_10053_gb300 import binding as B
    out = {"t": [], "h_density": [], "h_scalar": [], "max_speed": [], "max_mach": [], "newton_its": [],
           "gmres_its": []}
    t = 0.0
    with B.Grid(prob, precision=B.MIXED) as g:
        g.set_state(prob.U)
        if prob.q is not None:
            g.set_scalars(prob.q)
        g.autotune()
        t0 = time.perf_counter()
        for k in range(nsteps):
            st = g.step()
            t += st["dt"]
            if (k + 1) % every == 0 or k + 1 == nsteps:
                out["t"].append(t)
                diag = g.diagnostics()
                out["h_density"].append(diag["mixing_height"])
                out["max_speed"].append(diag["max_speed"])
                out["max_mach"].append(diag["max_mach"])
                out["h_scalar"].append(g.scalar_mixing_width() if prob.q is not None else None)
                out["newton_its"].append(st["newton_its"])
                out["gmres_its"].append(st["gmres_its"])
        out["wall_s"] = time.perf_counter() - t0
    out["steps"] = nsteps
    return out


def run_dt_study(n, t_end, cfls=(0.05, 10.0, 50.0)):
    """Sec. 5's time-step study at a smaller size: the Taylor-Green vortex to
    t_end with CFL_hydro fixed at the smallest value and capped at the larger
    ones; the mean kinetic energy over time for each (mixed precision)."""
    from paper_1610_10053_gb300 import binding as B
    from paper_1610_10053_gb300 import inputs as I
    out = {}
    for cfl in cfls:
        p = I.taylor_green(n=n).with_options(cfl=cfl)
        rec = {"t": [0.0], "kinetic_energy": [], "steps": 0, "newton_its": 0, "gmres_its": 0}
        with B.Grid(p, precision=B.MIXED) as g:
            g.set_state(p.U)
            rec["kinetic_energy"].append(g.diagnostics()["mean_kinetic_energy"])
            t, nrec = 0.0, 1
            t0 = time.perf_counter()
            while t < t_end * (1 - 1e-12):
                st = g.newton_step(t_end - t)  # the CFL step, capped at the end time
                t += st["dt"]
                rec["steps"] += 1
                rec["newton_its"] += st["newton_its"]
                rec["gmres_its"] += st["gmres_its"]
                if t >= nrec * t_end / 8 * (1 - 1e-12):
                    rec["t"].append(t)
                    rec["kinetic_energy"].append(g.diagnostics()["mean_kinetic_energy"])
                    nrec += 1
            rec["wall_s"] = time.perf_counter() - t0
        out["cfl_%g" % cfl] = rec
    return {"grid": "%d^3" % n, "t_end": t_end, "runs": out}


def run_convergence(n_max, t_end, n_min=64):
    """Sec. 4's grid-convergence study: the KH setup (no noise: a per-cell
    random seed differs between grids and cannot converge) run to t_end on
    n^2 grids, n = n_min .. n_max by doubling, each compared with the finest
    by the relative L1 error of the vertical velocity (mixed precision)."""
    from paper_1610_10053_gb300 import binding as B
    from paper_1610_10053_gb300 import inputs as I

    def run_to(n):
        p = I.kelvin_helmholtz(n=n, seed=2, noise=0.0)
        g = B.Grid(p, precision=B.MIXED)
        g.set_state(p.U)
        g.autotune()
        t, steps, t0 = 0.0, 0, time.perf_counter()
        while t < t_end * (1 - 1e-12):
            t += g.newton_step(t_end - t)["dt"]  # the CFL step, capped at the end time
            steps += 1
        return g, steps, time.perf_counter() - t0

    ref, steps, wall = run_to(n_max)
    out = {"t_end": t_end, "reference": "%d^2" % n_max, "reference_steps": steps, "reference_wall_s": wall,
           "n": [], "error": [], "steps": [], "wall_s": []}
    n = n_min
    while n < n_max:
        g, steps, wall = run_to(n)
        out["n"].append(n)
        out["error"].append(B.velocity_error(ref, g))
        out["steps"].append(steps)
        out["wall_s"].append(wall)
        g.close()
        n *= 2
    ref.close()
    e = out["error"]
    out["order"] = [math.log2(e[k] / e[k + 1]) for k in range(len(e) - 1)]
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(prob, label, steps=1):
    """The FP64 CPU oracle as it stands, on one implicit step of the same
    workload: on all host cores (its OpenMP build: loops over cells split
    over threads, reductions in fixed order, bitwise the serial results) and
    on one core."""
    from oracle import oracle as O
    O.build()
    model, ncpu = cpu_model(), os.cpu_count() or 1
    t0 = time.perf_counter()
    O.run(prob, nsteps=steps)
    el1 = time.perf_counter() - t0
    single = {"value": prob.ncells * steps / el1, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
              "sample": "%d implicit step(s) of %s (FP64, one thread), %.1f s" % (steps, label, el1)}
    if not O.openmp_available():
        single.update(cpu_model=model, single_thread=dict(single), note="no OpenMP runtime: one core only")
        return single
    with O.threaded(0) as nt:
        t0 = time.perf_counter()
        O.run(prob, nsteps=steps)
        eln = time.perf_counter() - t0
    return {"value": prob.ncells * steps / eln, "unit": "cell-steps/s", "cores": nt, "kind": "oracle",
            "sample": "%d implicit step(s) of %s (FP64, %d threads, OpenMP over cells), %.1f s"
                      % (steps, label, nt, eln),
            "cpu_model": model, "host_cpus": ncpu, "single_thread": single}



def run_reference(args):
    """The oracle (plain FP64 CPU solver) on the host cores, on the GPU arm's
    own workload: each step is one implicit step of the Kelvin-Helmholtz setup
    on the 512x512 grid, on all host cores (the oracle's OpenMP build)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1610_10053_gb300 import inputs as I
    O.build()
    prob = workload("kh512", 0)
    U = prob.U.copy()
    omp = O.openmp_available()
    ctx = O.threaded(0) if omp else contextlib.nullcontext(1)
    with ctx as nt:
        for _ in range(args.warmup):
            U, _ = O.run(prob, U=U, nsteps=1)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            U, _ = O.run(prob, U=U, nsteps=1)
            times.append(time.perf_counter() - t0)
    total = float(np.sum(times))
    value = prob.ncells * args.steps / total
    sample = ("each step: one implicit step of the same Kelvin-Helmholtz 512x512 workload (FP64 oracle, "
              "%d thread(s), OpenMP over cells); cell-steps/s is a rate" % nt)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["kh512"][0], "cells": prob.ncells, "precision": "fp64 (oracle)",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": nt, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="music", choices=["music", "reference"])
    ap.add_argument("--workload", default="kh512", choices=sorted(WORKLOADS))
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--series", type=int, default=0,
                    help="after the timed steps, run this many more recording the mixing widths")
    ap.add_argument("--every", type=int, default=100, help="record the series every this many steps")
    ap.add_argument("--dt-study", type=int, default=0,
                    help="also run the Taylor-Green time-step study on this many cells per edge")
    ap.add_argument("--dt-study-t", type=float, default=2.0, help="end time of the time-step study")
    ap.add_argument("--convergence", type=int, default=0,
                    help="also run the KH grid-convergence study up to this many cells per edge")
    ap.add_argument("--conv-t", type=float, default=0.5, help="end time of the convergence study")
    ap.add_argument("--serve-lane-cells", type=int, default=16384,
                    help="largest solve the server's batch lane takes in the lane-on rows")
    ap.add_argument("--serve-solves", type=int, default=256)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_music(args)


if __name__ == "__main__":
    main()
