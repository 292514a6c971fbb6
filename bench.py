#!/usr/bin/env python3
"""Throughput of the explicit finite-volume Euler residual + Runge-Kutta step
(SENSEI hot path, arXiv 2305.18057) on GB300, in cell-updates per second per
RK stage (interior cells x stages / time; the paper's ssspnt with np = 1 and
substeps counted is 1e-6 times this, Sec. 6 Eq. ssspnt).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3]
    python bench.py --impl reference ...     # the CPU oracle, timed on the host

One JSON line on rank 0.  A step is one full SSPRK3 step (ghost fill, time
step bound, three fused stencil/update stages, norm finalisation) over the
whole grid; the K timed steps run as one CUDA graph (--eager: launched one
by one).  With N > 1 (torchrun) every rank advances its own replica
of the grid on its own GPU: the method has no data-path exchange between
GPUs in this build ("replicas only"), so scaling is weak and the value is the
sum over ranks of the cells each advanced, over the slowest rank's time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage (FP64 vs mixed, at stated error); % HBM roofline"
UNIT = "cell-updates/s"

WORKLOADS = {
    # name: (builder, description)
    "c3": ("periodic3d 256^3: smooth curvilinear periodic map (5% of spacing), Mach 2.5 + 5 Fourier modes (1%), "
           "MUSCL van Leer + Roe (Harten 0.1), SSPRK3, CFL 0.5"),
    "c1": "advection2d 128^2: periodic box, Mach 2 at 30 deg + Gaussian bump, MUSCL minmod + Roe, SSPRK3, CFL 0.5",
    "c2": ("ramp2d 1024x512: 10-deg compression ramp, wall stretching 1.02, Mach 4 inflow (12270 Pa, 217 K), "
           "MUSCL van Leer + Roe, SSPRK3, CFL 0.5"),
    "c4": ("lattice3d: 4x4x4 blocks of seeded sizes in {32,48,64,96,128}, ramp-like grid, Mach 3 inflow, "
           "interface ghost exchange, MUSCL van Leer + Roe, SSPRK3, CFL 0.5"),
    "c5": ("ramp3d 512^3: 8-deg ramp extruded in k, wall stretching 1.005, Mach 4 inflow (12270 Pa, 217 K), "
           "MUSCL van Leer + Roe, SSPRK3, CFL 0.5"),
}

# Algorithmic FP64 operations per cell and stage of the fused stencil kernel
# (add, sub, mul = 1; fused multiply-add = 2; div, sqrt, rsqrt = 1; compares
# and sign tests 0), counted from the formulas the kernel evaluates: 3 Roe
# face fluxes (155 each), 3 directions of MUSCL face states (per limiter),
# the primitive variables (12), the flux-difference sum (25), the update
# (17, +10 on the stages that blend U^n) and the norm partials (20 on the
# first stage).  2D: 2 faces, 2 directions, residual sum 15.
ROE_FLOPS = 155
STATE_FLOPS = {"none": 25, "minmod": 30, "vanleer": 45}

# The same step as the oracle states it, counted by its op-counting build
# (oracle/opcount.cpp): operations per cell and RK stage over one SSPRK3 step
# (dt, three residuals and updates, norms) of the periodic 3D workload at
# 24^3, van Leer.  The plain oracle recomputes primitives for every face
# stencil, takes the limiter in its ratio form (a division per ratio) and
# normalises each face vector per call, so it performs about twice the
# kernel's operations; the kernel's own count above is the one the roofline
# uses (tests/test_oracle_opcount.py re-counts these numbers).
ORACLE_OPS_PER_CELL_STAGE = {"add": 682.894, "mul": 695.093, "div": 231.769, "sqrt": 10.708,
                             "cmp": 74.875, "abs": 117.771}


def alg_flops_per_cell(limiter, two_d, alpha_nonzero, first_stage):
    nd = 2 if two_d else 3
    f = nd * ROE_FLOPS + nd * STATE_FLOPS[limiter] + 12 + (15 if two_d else 25) + 17
    if alpha_nonzero:
        f += 10
    if first_stage:
        f += 20
    return f


def alg_bytes_per_cell(form, stage, two_d, stages=3):
    """Bytes the stencil kernel must move per interior cell in the launch of
    RK stage `stage` (0-based) of an SSPRK3 step:
      fp64: read U^(s-1) (40), write U^(s) (40), read U^n on the stages that
        blend it (40), FP64 face metrics (unit normal + area of the nd low
        faces, 32 B each) and 1/|Omega| (8), |Omega| (8) for the
        conservation sums on the first stage;
      fp32_flux: the same state bytes; the FP32 face-metric record of the
        tile-plane (13,952 B per 256 cells = 54.5 B, with 1/|Omega| in FP32)
        and the FP64 1/|Omega| (8) of the FP64 update;
      fp32_store: the record (54.5); first stage reads U (40) and writes D,
        X (20 + 20) and reads |Omega| (8); later stages read X (20), D (20),
        U^n (40) and write D, X (40) or, on the last, U (40)."""
    nd = 2 if two_d else 3
    rec = 13952.0 / 256.0
    if form == "fp32_store":
        return rec + (40 + 40 + 8 if stage == 0 else 40 + 40 + 40)
    if form == "fp32_flux":
        b = 40 + 40 + rec + 8
    else:
        b = 40 + 40 + nd * 32 + 8
    b += 40 if stage > 0 else 8
    return b


# DRAM bytes per interior cell and stencil launch, averaged over the three
# SSPRK3 stage launches, from ncu dram__bytes_read.sum + dram__bytes_write.sum
# of the 192^3 case of the periodic 3D workload (profiles/
# stencil_traffic_periodic3d_192.md for FP64, profiles/
# stencil32p_traffic_periodic3d_192.md for the FP32 forms); the same tile
# schedule at 256^3, so the traffic scales with the cells.  Re-measure when
# the kernel changes.
MEASURED_TRAFFIC_B_PER_CELL = {"fp64": 225.0, "fp32_flux": 184.0, "fp32_store": 172.5}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 vector peak derived from the unit counts: 152 SMs x 2 FP64 FMA lanes
# per SM per clock (the 1.25 TFLOP/s FP64 of GB300 at its 2070 MHz maximum
# clock) x 2 flops x clock.
def fp64_peak_tflops(sm_mhz=2070.0):
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


# FP32 vector peak derived the same way: 152 SMs x 128 FP32 FMA lanes per SM
# per clock x 2 flops x clock (80.5 TFLOP/s at 2070 MHz).
def fp32_peak_tflops(sm_mhz=2070.0):
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def step_flops_per_launch(limiter, two_d, cells, stages=3):
    """Formula flops of one stencil launch, averaged over the stages of an
    SSPRK3 step (the first accumulates the norm partials, the others blend
    U^n)."""
    return cells * (alg_flops_per_cell(limiter, two_d, False, True)
                    + alg_flops_per_cell(limiter, two_d, True, False) * (stages - 1)) / stages


def pipe_roofline(form, flops_per_launch, ms_per_launch):
    """The arithmetic side of a stencil launch's roofline: formula flops per
    mean launch time against the vector peak of the pipe that carries the
    reconstruction and the Roe flux -- FP64 for fp64; FP32 for the FP32 forms;
    for double-float (the FP64 formula carried as pairs of FP32 numbers on
    the FP32 pipe) the FP64 peak, so that a fraction above 1 is the factor by
    which it passes the native FP64 roof."""
    tf = flops_per_launch / (ms_per_launch / 1e3) / 1e12
    if form in ("fp32_flux", "fp32_store"):
        peak = fp32_peak_tflops(2070.0)
        src = "derived FP32 vector peak: 152 SMs x 128 FMA/clk x 2 flop x 2070 MHz"
    else:
        peak = fp64_peak_tflops(2070.0)
        src = "derived FP64 vector peak: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz"
        if form == "df64":
            src += " (double-float carries the FP64 formula on the FP32 pipe)"
    return {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
            "peak_source": src, "alg_flops_per_launch": flops_per_launch}


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), util=float(f[4]), hw=f[6], hwt=f[7], swt=f[8],
                                 pcap=f[9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r["util"] >= 50] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(load)}


# ------------------------------------------------------------- workloads --

def make_workload(name, n=None):
    from paper_2305_18057_gb300 import workloads as wl
    if name == "c3":
        return wl.periodic_3d(n=n or 256)
    if name == "c1":
        return wl.advection_2d(n=128)
    if name == "c2":
        return wl.ramp_2d(ni=1024, nj=512)
    if name == "c4":
        return wl.lattice_3d()
    if name == "c5":
        return wl.ramp_3d(n=n or 512)
    raise SystemExit(f"unknown workload {name}")


def gpu_setup(w, precision, tune=True):
    """Grid, states and (tune) the autotuned schedule (kchunk, persistent)."""
    import torch
    from paper_2305_18057_gb300 import sensei, workloads as wl
    g = sensei.Grid(w.dims, w.nodes, gamma=w.gamma, limiter=wl.LIMITERS[w.limiter], kappa=w.kappa, eps=w.eps,
                    entropy_fix=w.fix, precision=precision, mu=w.mu, prandtl=w.prandtl)
    for b, faces in enumerate(w.bcs):
        for f in range(4 if w.dims[b][2] == 1 else 6):
            bc = faces[f]
            g.set_bc(b, f, bc.type, bc.prim, bc.nbr, bc.nbr_face)
    Us = []
    for b in range(len(w.dims)):
        U = g.new_state(b)
        g.upload(U, b, w.U0[b])
        Us.append(U)
    schedule = g.autotune(Us) if tune else None
    torch.cuda.synchronize()
    return g, Us, schedule


def time_graph(g, Us, steps, rk, cfl):
    """K consecutive steps as one CUDA graph (sensei_steps_graph_create: on
    the 3D mixed-precision grids every step after the first takes its CFL
    bound from the last stage of the step before), replayed once to warm up
    and once timed; returns ms for the K steps."""
    import torch
    graph = g.steps_graph(Us, steps, rk, cfl=cfl)
    graph.launch()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    graph.launch()
    e1.record(s)
    torch.cuda.synchronize()
    graph.close()
    return e0.elapsed_time(e1)


def time_steps(g, Us, steps, rk, cfl, profile=False):
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if profile:
        g.profile(True)
        g.profile_read(reset=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(steps):
        g.rk_step(Us, rk, cfl=cfl)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = None
    if profile:
        # stencil launch times by Runge-Kutta stage (the grid's launches cycle
        # through the stages in order)
        per = g.profile_launches()
        st_ms, st_n, k_n = g.profile_read(reset=True)
        g.profile(False)
        nst = len(per) // max(steps, 1)
        by_stage = [sum(per[i::nst]) / len(per[i::nst]) for i in range(nst)] if nst else []
        prof = (st_ms, st_n, k_n, by_stage)
    return ms, prof


# --------------------------------------------------------------- reference --

# k extent of the single-block 3D sample every oracle leg times (the
# cpu_baseline legs and the --impl reference arm use the same slab)
ORACLE_SAMPLE_DEPTH = {"c3": 48, "c5": 12}


def oracle_sample(w_name, steps, warmup, depth=None, threads=1):
    """Time the CPU oracle as it stands on `threads` host threads (its
    OpenMP loops over k-planes; the results are bitwise those of one
    thread) on a bounded sample of the workload: for the single-block 3D
    workloads the same grid family with `depth` cells in k (k-periodic; the
    per-cell cost does not depend on the k extent), a lattice of smaller
    blocks for the multiblock one, the 2D grids whole or in part.  Returns
    (cell-updates/s, seconds, sample description, cells, threads used)."""
    import numpy as np
    import oracle
    from paper_2305_18057_gb300 import workloads as wl
    w = make_workload(w_name) if w_name in ("c1",) else None
    depth = depth or ORACLE_SAMPLE_DEPTH.get(w_name)
    if w_name == "c3":
        w = wl.periodic_3d(n=256, nk=depth)
        sample = f"SSPRK3 steps of the 256x256x{depth} grid of the periodic 3D family (same generator and state recipe)"
    elif w_name == "c5":
        w = wl.ramp_3d(ni=512, nj=512, nk=depth)
        sample = f"SSPRK3 steps of the 512x512x{depth} grid of the 3D ramp family (k-periodic)"
    elif w_name == "c4":
        w = wl.lattice_3d(sizes=(16, 24, 32))
        sample = "SSPRK3 steps of the 4x4x4 lattice with block sizes drawn from {16,24,32}"
    elif w_name == "c2":
        w = wl.ramp_2d(ni=1024, nj=128)
        sample = "SSPRK3 steps of a 1024x128 (near-wall quarter) version of the 1024x512 ramp grid"
    else:
        sample = "SSPRK3 steps of the whole 128^2 grid"
    og = oracle.OracleGrid(w.dims, w.nodes, gamma=w.gamma, limiter=wl.LIMITERS[w.limiter], kappa=w.kappa,
                           eps=w.eps, fix=w.fix)
    for b, faces in enumerate(w.bcs):
        for f in range(4 if w.dims[b][2] == 1 else 6):
            bc = faces[f]
            og.set_bc(b, f, bc.type, bc.prim, bc.nbr, bc.nbr_face)
    Us = []
    for b in range(len(w.dims)):
        U = og.alloc_state(b)
        og.interior(U, b)[...] = w.U0[b]
        Us.append(U)
    used = oracle.set_threads(threads)
    try:
        for _ in range(warmup):
            og.rk_step(Us, oracle.RK3_SSP, cfl=w.cfl)
        t0 = time.perf_counter()
        for _ in range(steps):
            og.rk_step(Us, oracle.RK3_SSP, cfl=w.cfl)
        t = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    cells = sum(a * b * c for a, b, c in w.dims)
    return cells * 3 * steps / t, t, f"{steps} {sample}", cells, used


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    value, secs, sample, cells, used = oracle_sample(args.workload, args.steps, args.warmup,
                                                     threads=os.cpu_count() or 1)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_for(args.workload),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name") and line.split(":", 1)[1].strip() not in ("-", ""):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def aggregate_ranks(ms, units, device):
    """Whole-job figures over the ranks of the default process group: the
    slowest rank's time (ms) and the sum of the cell updates every rank
    performed.  Every rank calls it (a collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item()


def config_for(name):
    return {"workload": WORKLOADS[name], "l2": "inputs larger than L2 (state >= 0.7 GB)" if name in ("c3", "c4", "c5")
            else "inputs L2-resident (noted, not an HBM claim)", "parallelism": "replicas"}


# ------------------------------------------------------------ C4 lattice --

def lattice_variant(args, peaks, peak_src, world):
    """The batched multiblock form inside the default run: the 64-block
    lattice (uneven blocks, interface ghost exchange) in FP32 flux on the
    FP64 state, one batched launch per RK stage over all blocks, one CUDA
    graph of the timed steps, autotuned schedule; beside it the plain FP64 form on the same
    lattice (its speedup) and the density error against it after the same
    steps from the same state."""
    from paper_2305_18057_gb300 import workloads as wl
    out = workload_variant(args, peaks, peak_src, world, wl.lattice_3d(), "fp32_flux", max(3, min(args.steps, 10)))
    out["workload"] = WORKLOADS["c4"]
    return out


def ramp_variant(args, peaks, peak_src, world):
    """The 512^3 Mach-4 ramp (one block, wall / inflow / outflow rules,
    stretched grid) inside the default run: the FP32-storage form, one CUDA
    graph of the timed steps, autotuned schedule; beside it the FP64 form
    (its speedup and the density error against it)."""
    from paper_2305_18057_gb300 import workloads as wl
    out = workload_variant(args, peaks, peak_src, world, wl.ramp_3d(n=512), "fp32_store", 5)
    out["workload"] = WORKLOADS["c5"]
    return out


def workload_variant(args, peaks, peak_src, world, w, form, steps):
    """One mixed-precision form on workload w: CUDA-graph steps with the
    autotuned schedule, its stencil roofline, and the FP64 form on the same
    workload (speedup, density error after the same steps from the same
    state)."""
    import torch
    from paper_2305_18057_gb300 import sensei
    cells, stages, rk = w.cells, 3, sensei.RK3_SSP
    res = {}
    states = {}
    precs = {"fp32_flux": sensei.FP32_FLUX, "fp32_store": sensei.FP32_STORE}
    kernels = {"fp32_flux": "stencil32p_kernel<double> (paired FP32 MUSCL + Roe on the FP64 state)",
               "fp32_store": "stencil32p_kernel<float> / <double> (paired FP32 MUSCL + Roe, FP32 stage states)"}
    for name, prec in (("fp64", sensei.FP64), (form, precs[form])):
        g, Us, sched = gpu_setup(w, prec)
        for _ in range(args.warmup):
            g.rk_step(Us, rk, cfl=w.cfl)
        torch.cuda.synchronize()
        ms = time_graph(g, Us, steps, rk, w.cfl)
        _, prof = time_steps(g, Us, 3, rk, w.cfl, profile=True)
        per_launch = prof[0] / max(prof[1], 1)
        r = {"value": cells * stages * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
             "schedule": g.schedule(), "kernel_ms_per_launch": per_launch,
             "steps": steps, "step": "one cuda graph of the K steps"}
        if name == form:
            byts = cells * sum(alg_bytes_per_cell(form, s_, False) for s_ in range(stages)) / stages
            hbm = byts / (per_launch / 1e3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": hbm / peaks["hbm_gbs"], "peak_source": peak_src,
                             "kernel": kernels[form],
                             "alg_bytes_per_launch": byts, "kernel_ms_per_launch": per_launch,
                             "kernel_ms_by_stage": prof[3],
                             "pipe": pipe_roofline(form, step_flops_per_launch(w.limiter, False, cells, stages),
                                                   per_launch)}
        res[name] = r
        # the same number of steps from the initial state for the error
        for b in range(len(w.dims)):
            g.upload(Us[b], b, w.U0[b])
        for _ in range(steps):
            g.rk_step(Us, rk, cfl=w.cfl)
        torch.cuda.synchronize()
        states[name] = [g.interior_view(Us[b], b)[0].clone() for b in range(len(w.dims))]
        del g, Us
        torch.cuda.empty_cache()
    num = math.sqrt(sum(float(torch.linalg.vector_norm(a - b_)) ** 2
                        for a, b_ in zip(states[form], states["fp64"])))
    den = math.sqrt(sum(float(torch.linalg.vector_norm(b_)) ** 2 for b_ in states["fp64"]))
    out = dict(res[form])
    out.update({
        "cells": cells, "blocks": len(w.dims), "precision": form,
        "speedup_vs_fp64": (res[form]["value"] / res["fp64"]["value"]) if world == 1 else None,
        "rho_l2_rel_err_vs_fp64": num / den, "steps_compared": steps,
        "fp64": res["fp64"]})
    return out


# --------------------------------------------------------- co-execution --

def hetero_study(args):
    """NEXT row f4 measured: the 256^3 periodic workload split into k-slabs
    between the GPU and the host worker on all host cores (Sec. 4), over a
    sweep of host shares, against the GPU alone, beside the prediction of
    Eq. hete from the two speeds measured separately (alpha = 0: the
    interior term; the exchange is measured, not modelled)."""
    import torch
    from paper_2305_18057_gb300 import sensei, workloads as wl
    w = wl.periodic_3d(n=args.n or 256)
    ni, nj, nk = w.dims[0]
    cells = w.cells
    threads = os.cpu_count() or 1
    rk, steps, warm = sensei.RK3_SSP, 4, 2
    bcs = [(bc.type, bc.prim) for bc in w.bcs[0]]
    # the GPU alone, eager steps (the driver launches eagerly too)
    g, Us, _ = gpu_setup(w, sensei.FP64, tune=False)
    for _ in range(warm):
        g.rk_step(Us, rk, cfl=w.cfl)
    ms_gpu, _ = time_steps(g, Us, steps, rk, w.cfl)
    del g, Us
    torch.cuda.empty_cache()
    G = cells * 3 * steps / (ms_gpu / 1e3)
    # the host worker alone on a k-slab of the same grid (all cores)
    slab = 16
    hb = sensei.HostBlock((ni, nj, slab), np.ascontiguousarray(w.nodes[0][:, :slab + 1]),
                          limiter=wl.LIMITERS[w.limiter], entropy_fix=w.fix, threads=threads)
    for f in range(6):
        hb.set_bc(f, sensei.BC_PERIODIC)
    hb.interior()[...] = w.U0[0][:, :slab]
    dt = hb.dt_min(w.cfl)
    hb.step(rk, dt)
    t0 = time.perf_counter()
    for _ in range(2):
        hb.step(rk, dt)
    C = ni * nj * slab * 3 * 2 / (time.perf_counter() - t0)
    hb.close()
    rows = []
    for nk_host in (4, 8, 12, 16, 24, 32):
        h = sensei.Hetero(w.dims[0], w.nodes[0], bcs, nk_host, threads, limiter=wl.LIMITERS[w.limiter],
                          entropy_fix=w.fix)
        h.upload(w.U0[0])
        for _ in range(warm):
            h.step(rk, cfl=w.cfl)
        tot = np.zeros(4)
        for _ in range(steps):
            _, t = h.step(rk, cfl=w.cfl)
            tot += np.array(t)
        h.close()
        torch.cuda.empty_cache()
        ms = tot[0] / steps
        share = nk_host / nk
        pred_ms = max((1 - share) * cells * 3 / G, share * cells * 3 / C) * 1e3
        rows.append({"nk_host": nk_host, "host_share": share, "ms_per_step": ms,
                     "speedup_vs_gpu_only": (ms_gpu / steps) / ms, "gpu_stage_ms": tot[1] / steps,
                     "host_stage_ms": tot[2] / steps, "exchange_ms": tot[3] / steps,
                     "model_ms": pred_ms, "model_speedup": (ms_gpu / steps) / pred_ms,
                     # Eq. hete's alpha term taken as the measured exchange
                     "model_with_exchange_ms": pred_ms + tot[3] / steps})
    best = max(rows, key=lambda r: r["speedup_vs_gpu_only"])
    return {
        "workload": WORKLOADS["c3"] if not args.n else f"periodic3d {args.n}^3",
        "split": "k-slabs: the last nk_host planes on the host worker (all host cores, OpenMP over (k, j) rows), "
                 "the rest on the GPU (default schedule, eager stages); the two cut faces (periodic wrap) exchanged "
                 "through pinned host memory every RK stage",
        "host_threads": threads, "gpu_only_ms_per_step": ms_gpu / steps,
        "gpu_cell_updates_per_s": G, "host_cell_updates_per_s": C, "r_gc": G / C,
        "model": "Eq. hete with alpha = 0: T = max(N_g / G, N_c / C); optimum share C / (G + C), "
                 "speedup (G + C) / G (ideal overlap, exchange not modelled)",
        "model_best_share": C / (G + C), "model_best_speedup": (G + C) / G,
        "measured_best": {"nk_host": best["nk_host"], "speedup_vs_gpu_only": best["speedup_vs_gpu_only"]},
        "sweep": rows}


# ------------------------------------------------------------ oracle leg --
# The CPU-baseline leg: the only part of the bench that runs the oracle
# (rank 0, one GPU, after every timed region).  It times the oracle on one
# host core and on all of them, on the same slab as the --impl reference
# arm, and states the error of every GPU result against the oracle.

def _core_boxes(w, margin=6, core=10):
    """(block, lo, hi) of sampled sub-boxes (core + 2 margin cells per side)
    for the one-step comparison: strictly inside the block for the periodic
    grid and the lattice; for the single-block ramp also boxes on its
    inflow, wall, outflow and periodic faces."""
    e = core + 2 * margin
    boxes = []
    if len(w.dims) > 1:
        # lattice: boxes well inside four blocks (no interface face touched)
        for b in (0, 21, 42, 63):
            ni, nj, nk = w.dims[b]
            lo = ((ni - e) // 2, (nj - e) // 2, (nk - e) // 2)
            boxes.append((b, lo, (lo[0] + e, lo[1] + e, lo[2] + e)))
        return boxes
    ni, nj, nk = w.dims[0]
    starts = [(0, 0, 0), (ni - e, nj - e, nk - e), (ni // 2 - e // 2, 3, nk - e - 5), (7, nj // 3, nk // 2)]
    starts = [tuple(max(0, min(a, n - e)) for a, n in zip(st, (ni, nj, nk))) for st in starts]
    # a 2D block (one plane) keeps its single plane: the box spans k = 0 .. 1
    return [(0, st, (st[0] + e, st[1] + e, st[2] + e if nk > 1 else 1)) for st in starts]


def _oracle_subbox_step(w, b, lo, hi, dt, margin=6):
    """One oracle SSPRK3 step with the given dt on the cells lo <= (i,j,k) <
    hi of block b of the workload's initial state; the ghosts of cut faces
    are copied from the state (wrapped across periodic faces), those of the
    block's own non-periodic faces follow its rule.  Returns the (5, ...)
    states before and after on the box's core (margin cells inside)."""
    import oracle
    from paper_2305_18057_gb300 import workloads as wl
    ni, nj, nk = w.dims[b]
    (i0, j0, k0), (i1, j1, k1) = lo, hi
    faces = w.bcs[b]
    X = np.ascontiguousarray(w.nodes[b][:, k0:k1 + 1, j0:j1 + 1, i0:i1 + 1])
    g = oracle.OracleGrid([(i1 - i0, j1 - j0, k1 - k0)], [X], gamma=w.gamma, limiter=wl.LIMITERS[w.limiter],
                          kappa=w.kappa, eps=w.eps, fix=w.fix, mu=w.mu, prandtl=w.prandtl)

    def rng(a0, a1, n, periodic):
        r = np.arange(a0 - oracle.NG, a1 + oracle.NG)
        return r % n if periodic else np.clip(r, 0, n - 1)

    per = [faces[2 * d].type == wl.PERIODIC for d in range(3)]
    ii, jj = rng(i0, i1, ni, per[0]), rng(j0, j1, nj, per[1])
    kk = rng(k0, k1, nk, per[2]) if nk > 1 else np.zeros(1, dtype=np.int64)   # 2D: no k ghosts
    U = np.ascontiguousarray(w.U0[b][:, kk[:, None, None], jj[None, :, None], ii[None, None, :]])
    on_face = [i0 == 0, i1 == ni, j0 == 0, j1 == nj, k0 == 0, k1 == nk]
    for f in range(6 if nk > 1 else 4):
        bc = faces[f]
        if on_face[f] and bc.type not in (wl.PERIODIC, wl.INTERFACE):
            g.set_bc(0, f, bc.type, bc.prim)
    g.fill_ghosts([U])
    m = margin
    ks = slice(m, -m) if nk > 1 else slice(None)
    before = g.interior(U, 0)[:, ks, m:-m, m:-m].copy()
    g.rk_step([U], oracle.RK3_SSP, dt=dt)
    return before, g.interior(U, 0)[:, ks, m:-m, m:-m].copy()


def _gpu_one_step(w, precision, boxes, dt, margin=6):
    """The GPU path of one precision form: one SSPRK3 step with the given dt
    from the workload's initial state; the box cores after the step."""
    import torch
    from paper_2305_18057_gb300 import sensei
    g, Us, _ = gpu_setup(w, precision, tune=False)
    if dt is None:
        dt_t = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
        g.rk_step(Us, sensei.RK3_SSP, cfl=w.cfl, dt_used=dt_t)
        dt = float(dt_t.item())
    else:
        g.rk_step(Us, sensei.RK3_SSP, cfl=0.0, dt=dt)
    torch.cuda.synchronize()
    m = margin
    out = []
    for b, lo, hi in boxes:
        mk = m if w.dims[b][2] > 1 else 0
        v = g.interior_view(Us[b], b)[:, lo[2] + mk:hi[2] - mk, lo[1] + m:hi[1] - m, lo[0] + m:hi[0] - m]
        out.append(v.cpu().numpy().copy())
    del g, Us
    torch.cuda.empty_cache()
    return out, dt


def _err_table(got, want, before):
    """Per conserved variable (rho, rho u, rho v, rho w, rho e_t): relative L2
    and max error of the state after the step, and of its increment over the
    step, against the oracle's, over every sampled cell.  A variable's
    scale is floored at 1e-3 of the largest variable's (a component that is
    near zero everywhere is measured against the flow's scale)."""
    g = np.concatenate([x.reshape(5, -1) for x in got], axis=1)
    o = np.concatenate([x.reshape(5, -1) for x in want], axis=1)
    u0 = np.concatenate([x.reshape(5, -1) for x in before], axis=1)

    def rel(a, b):
        l2n = np.sqrt((b * b).sum(axis=1))
        mxn = np.abs(b).max(axis=1)
        l2n = np.maximum(l2n, 1e-3 * l2n.max())
        mxn = np.maximum(mxn, 1e-3 * mxn.max())
        return (np.sqrt(((a - b) ** 2).sum(axis=1)) / l2n).tolist(), (np.abs(a - b).max(axis=1) / mxn).tolist()

    l2, mx = rel(g, o)
    out = {"vars": ["rho", "rho_u", "rho_v", "rho_w", "rho_e_t"], "l2": l2, "max": mx}
    d = o - u0
    if np.abs(d).max() > 1e-12 * np.abs(o).max():
        out["increment_l2"], out["increment_max"] = rel(g - u0, d)
    return out


def err_vs_oracle(w, forms):
    """{form: error table} of one SSPRK3 step of each precision form against
    the oracle's step on sampled sub-box cores (the same dt for all: the
    FP64 path's CFL dt, itself checked against the oracle's to 1e-14 by the
    tests)."""
    from paper_2305_18057_gb300 import sensei
    boxes = _core_boxes(w)
    got64, dt = _gpu_one_step(w, sensei.FP64, boxes, None)
    res = [_oracle_subbox_step(w, b, lo, hi, dt) for b, lo, hi in boxes]
    before = [r[0] for r in res]
    want = [r[1] for r in res]
    core = [tuple(h - l - 12 for l, h in zip(lo, hi)) for _, lo, hi in boxes]
    sample = (f"one SSPRK3 step (dt {dt:.6g}, the FP64 path's CFL step) from the initial state, on the cores "
              f"{core[0][0]}^{3 if w.dims[boxes[0][0]][2] > 1 else 2} of {len(boxes)} sub-boxes (6 margin cells; "
              f"the oracle on each sub-box with the "
              f"state as the ghosts of its cut faces)")
    out = {}
    for name, prec in forms:
        got = got64 if prec == sensei.FP64 else _gpu_one_step(w, prec, boxes, dt)[0]
        t = _err_table(got, want, before)
        t["sample"] = sample
        out[name] = t
    return out


def oracle_leg(args, w, line, main_prec):
    from paper_2305_18057_gb300 import sensei
    ncpu = os.cpu_count() or 1
    steps = 3 if args.workload in ("c3", "c5") else 2
    v1, s1, sample, _, _ = oracle_sample(args.workload, steps, 0, threads=1)
    va, sa, _, _, used = oracle_sample(args.workload, steps, 0, threads=ncpu)
    line["cpu_baseline"] = {"value": va, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                            "seconds": sa, "cpu": cpu_model(), "host_cpus": ncpu,
                            "one_core": {"value": v1, "cores": 1, "seconds": s1},
                            "note": "the oracle as it stands; all cores run its OpenMP loops over k-planes "
                                    "(bitwise the one-core results); the --impl reference arm times the same slab"}
    forms = [("fp64", sensei.FP64), ("fp32_flux", sensei.FP32_FLUX), ("fp32_store", sensei.FP32_STORE),
             ("df64", sensei.DF64)]
    if args.workload == "c4":
        forms = forms[:2]
    w_err = w
    if args.workload == "c5":
        # the ramps (3D here, 2D below) start as a uniform inflow, so the
        # sampled cores (away from the wall) have zero increments: the
        # comparison takes seeded 5% perturbations of rho, p and u on the
        # same grid
        from paper_2305_18057_gb300 import workloads as wl
        w_err = wl.ramp_3d(n=w.dims[0][0], perturb=0.05)
    elif args.workload == "c2":
        from paper_2305_18057_gb300 import workloads as wl
        w_err = wl.ramp_2d(ni=w.dims[0][0], nj=w.dims[0][1], perturb=0.05)
    elif args.workload == "c4":
        # the lattice's uniform inflow likewise
        from paper_2305_18057_gb300 import workloads as wl
        w_err = wl.lattice_3d(perturb=0.05)
    table = err_vs_oracle(w_err, forms)
    if w_err is not w:
        for t in table.values():
            t["sample"] += "; the workload's state with seeded 5% perturbations"
    main_name = "fp64" if main_prec == sensei.FP64 else "fp32_flux"
    line["err_vs_oracle"] = table[main_name]
    for name, t in table.items():
        if name in line.get("variants", {}):
            line["variants"][name]["err_vs_oracle"] = t
    vis = line.get("variants", {}).get("fp64_viscous")
    if vis is not None:
        # the Navier-Stokes form against the oracle's viscous flux, same sampling
        import dataclasses
        wv = dataclasses.replace(w_err, mu=vis["mu"], prandtl=vis["prandtl"])
        tv = err_vs_oracle(wv, [("fp64_viscous", sensei.FP64)])["fp64_viscous"]
        tv["sample"] += "; the Navier-Stokes form (mu of Re 1000)"
        vis["err_vs_oracle"] = tv
    if "c4_lattice" in line.get("variants", {}):
        # the lattice's initial state is a uniform inflow, whose residual
        # vanishes inside the blocks: the comparison takes it with seeded 5%
        # perturbations of rho, p and u so that every sampled cell moves
        from paper_2305_18057_gb300 import workloads as wl
        t4 = err_vs_oracle(wl.lattice_3d(perturb=0.05), [("fp64", sensei.FP64), ("fp32_flux", sensei.FP32_FLUX)])
        for t in t4.values():
            t["sample"] += "; the lattice's state with seeded 5% perturbations"
        line["variants"]["c4_lattice"]["err_vs_oracle"] = t4["fp32_flux"]
        line["variants"]["c4_lattice"]["fp64"]["err_vs_oracle"] = t4["fp64"]
    if "c5_ramp" in line.get("variants", {}):
        # the ramp's uniform inflow likewise: seeded 5% perturbations
        from paper_2305_18057_gb300 import workloads as wl
        t5 = err_vs_oracle(wl.ramp_3d(n=512, perturb=0.05), [("fp64", sensei.FP64), ("fp32_store", sensei.FP32_STORE)])
        for t in t5.values():
            t["sample"] += "; the ramp's state with seeded 5% perturbations"
        line["variants"]["c5_ramp"]["err_vs_oracle"] = t5["fp32_store"]
        line["variants"]["c5_ramp"]["fp64"]["err_vs_oracle"] = t5["fp64"]


# -------------------------------------------------------------------- main --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-perf-model", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="grid size override (c3, c5): small profiling cases")
    ap.add_argument("--eager", action="store_true",
                    help="time eager launches instead of CUDA-graph replays of the step")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2305_18057_gb300 import build as libbuild
    from paper_2305_18057_gb300 import sensei
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if rank == 0 or world == 1:
        libbuild.build()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        libbuild.build()
    torch.cuda.set_device(local)
    sensei.load()

    w = make_workload(args.workload, args.n)
    two_d = all(d[2] == 1 for d in w.dims)
    cells = w.cells
    rk = sensei.RK3_SSP
    stages = 3
    # the batched multiblock workload runs FP32 flux on the FP64 state, the
    # others FP64 (mixed forms as variants); the main line replays a CUDA
    # graph of one step
    main_prec = sensei.FP32_FLUX if args.workload == "c4" else sensei.FP64
    use_graph = not args.eager
    g, Us, schedule = gpu_setup(w, main_prec)
    for _ in range(args.warmup):
        g.rk_step(Us, rk, cfl=w.cfl)
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = vis.split(",")[local] if vis else str(local)
    clocks = ClockSampler(gpu_index)
    if world > 1:
        dist.barrier()
    clocks.start()
    time.sleep(0.4)
    if use_graph:
        ms = time_graph(g, Us, args.steps, rk, w.cfl)
        clk = clocks.stop()
        # kernel times for the roofline from an eager, instrumented pass
        _, prof = time_steps(g, Us, max(3, min(args.steps, 5)), rk, w.cfl, profile=True)
        prof = (prof[0], prof[1], prof[2] * args.steps // max(3, min(args.steps, 5)), prof[3])
    else:
        ms, prof = time_steps(g, Us, args.steps, rk, w.cfl, profile=True)
        clk = clocks.stop()
    units = cells * stages * args.steps
    if world > 1:
        ms, units = aggregate_ranks(ms, units, "cuda")
    value = units / (ms / 1e3)

    # the dominant kernel: the fused stencil/update kernel
    st_ms, st_n, k_launches, by_stage = prof
    per_launch_ms = st_ms / max(st_n, 1)
    peaks, peak_src = measured_peaks()
    form = "fp64" if main_prec == sensei.FP64 else "fp32_flux"
    byts = cells * sum(alg_bytes_per_cell(form, s_, two_d) for s_ in range(stages)) / stages
    hbm_gbs = byts / (per_launch_ms / 1e3) / 1e9
    if main_prec == sensei.FP64:
        flops = step_flops_per_launch(w.limiter, two_d, cells, stages)
        fp64_peak = fp64_peak_tflops(2070.0)
        achieved_tf = flops / (per_launch_ms / 1e3) / 1e12
        roofline = {
            "bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved_tf / fp64_peak,
            "traffic": None if two_d else MEASURED_TRAFFIC_B_PER_CELL["fp64"] * cells,
            "traffic_source": "ncu DRAM bytes per cell of the 192^3 capture x cells (3-stage average)",
            "kernel": "stencil_kernel<double,double> (fused MUSCL + Roe + residual + RK stage)",
            "peak_source": "derived FP64 vector peak: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz",
            "alg_flops_per_launch": flops, "kernel_ms_per_launch": per_launch_ms, "kernel_ms_by_stage": by_stage,
            "oracle_ops_per_cell_stage": ORACLE_OPS_PER_CELL_STAGE,
            "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": peaks["hbm_gbs"], "frac": hbm_gbs / peaks["hbm_gbs"],
                    "peak_source": peak_src, "alg_bytes_per_launch": byts},
        }
    else:
        roofline = {
            "bound": "hbm", "achieved": hbm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": hbm_gbs / peaks["hbm_gbs"],
            "traffic": None if two_d else MEASURED_TRAFFIC_B_PER_CELL["fp32_flux"] * cells,
            "traffic_source": "ncu DRAM bytes per cell of the 192^3 capture x cells (3-stage average)",
            "peak_source": peak_src,
            "kernel": "stencil32p_kernel<double> (paired FP32 MUSCL + Roe on the FP64 state, FP64 update)",
            "alg_bytes_per_launch": byts, "kernel_ms_per_launch": per_launch_ms, "kernel_ms_by_stage": by_stage,
            "pipe": pipe_roofline(form, step_flops_per_launch(w.limiter, two_d, cells, stages), per_launch_ms),
        }

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if main_prec == sensei.FP64 else "f32 flux / f64 state", "data": "synthetic",
        "config": dict(config_for(args.workload), cells=cells, blocks=len(w.dims),
                       schedule={"kchunk": schedule[0], "persistent": schedule[1]},
                       step="one cuda graph of the K steps" if use_graph else "eager launches"),
        "ssspnt": value * 1e-6, "gpu_launches": k_launches, "roofline": roofline, "clocks": clk,
    }

    # end to end through the C ABI with host buffers: every step copies the
    # state in from pinned host memory, steps, copies the new state and the
    # norms back
    Uh = [torch.empty(U.numel(), dtype=torch.float64, pin_memory=True) for U in Us]
    for a, b_ in zip(Uh, Us):
        a.copy_(b_)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.steps):
        for a, b_ in zip(Uh, Us):
            b_.copy_(a, non_blocking=True)
        g.rk_step(Us, rk, cfl=w.cfl)
        for a, b_ in zip(Uh, Us):
            a.copy_(b_, non_blocking=True)
        g.norms()
    e1.record(s)
    torch.cuda.synchronize()
    ems = e0.elapsed_time(e1)
    if world > 1:
        ems, _ = aggregate_ranks(ems, 0, "cuda")
    state_bytes = sum(U.numel() * 8 for U in Us)
    line["e2e"] = {"value": units / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                   "d2h_bytes_per_step": state_bytes + 15 * 8}

    # the mixed-precision forms on the same workload: FP32 reconstruction and
    # flux on the FP64 state (fp32_flux), and additionally FP32 stage storage
    # with the FP64 accumulation U^{n+1} = U^n + D (fp32_store); error vs the
    # FP64 path (itself matched to the oracle) after the same steps from the
    # same state
    if not args.no_variants:
        n_cmp = args.warmup + args.steps
        g64, U64, _ = gpu_setup(w, sensei.FP64, tune=False)
        for _ in range(n_cmp):
            g64.rk_step(U64, rk, cfl=w.cfl)
        torch.cuda.synchronize()
        line["variants"] = {}
        for vname, prec in (("fp64", sensei.FP64), ("fp32_flux", sensei.FP32_FLUX),
                            ("fp32_store", sensei.FP32_STORE), ("df64", sensei.DF64)):
            if prec == main_prec:
                continue
            gv, Uv, sched_v = gpu_setup(w, prec)
            for _ in range(args.warmup):
                gv.rk_step(Uv, rk, cfl=w.cfl)
            torch.cuda.synchronize()
            msv = time_graph(gv, Uv, args.steps, rk, w.cfl)
            _, profv = time_steps(gv, Uv, max(3, min(args.steps, 5)), rk, w.cfl, profile=True)
            # the FP64 path's number of steps from the same initial state
            for b in range(len(w.dims)):
                gv.upload(Uv[b], b, w.U0[b])
            for _ in range(n_cmp):
                gv.rk_step(Uv, rk, cfl=w.cfl)
            torch.cuda.synchronize()
            errs = []
            for b in range(len(w.dims)):
                a64 = g64.interior_view(U64[b], b)
                av = gv.interior_view(Uv[b], b)
                errs.append((float(torch.linalg.vector_norm(av[0] - a64[0])),
                             float(torch.linalg.vector_norm(a64[0]))))
            rho_l2 = math.sqrt(sum(e[0] ** 2 for e in errs)) / math.sqrt(sum(e[1] ** 2 for e in errs))
            vv = cells * stages * args.steps / (msv / 1e3)
            stv = profv[0] / max(profv[1], 1)
            bv = cells * sum(alg_bytes_per_cell("fp64" if vname == "df64" else vname, s_, two_d)
                             for s_ in range(stages)) / stages
            line["variants"][vname] = {
                "value": vv, "unit": UNIT, "ms_per_step": msv / args.steps,
                "speedup_vs_fp64": (vv / value if main_prec == sensei.FP64 else None) if world == 1 else None,
                "schedule": {"kchunk": sched_v[0], "persistent": sched_v[1]},
                "rho_l2_rel_err_vs_fp64": rho_l2, "steps_compared": n_cmp,
                "roofline": {"bound": "hbm", "achieved": bv / (stv / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                             "unit": "GB/s", "frac": bv / (stv / 1e3) / 1e9 / peaks["hbm_gbs"],
                             "kernel_ms_per_launch": stv, "kernel_ms_by_stage": profv[3],
                             "traffic": (MEASURED_TRAFFIC_B_PER_CELL[vname] * cells
                                         if not two_d and vname in MEASURED_TRAFFIC_B_PER_CELL else None),
                             "alg_bytes_per_launch": bv, "peak_source": peak_src,
                             "pipe": pipe_roofline(vname, step_flops_per_launch(w.limiter, two_d, cells, stages),
                                                   stv)}}
            del gv, Uv
        del g64, U64
        # the Navier-Stokes form (NEXT row f2) in FP64 on the same grid and
        # state, with the viscosity of a Reynolds number of 1000 on the mean
        # speed and density and a unit length
        import dataclasses
        speed = float(np.sqrt(sum(float(np.mean(w.U0[0][a] / w.U0[0][0])) ** 2 for a in (1, 2, 3))))
        rho_m = float(np.mean(w.U0[0][0]))
        mu = rho_m * speed / 1000.0
        wv = dataclasses.replace(w, mu=mu)
        gv, Uv, sched_v = gpu_setup(wv, sensei.FP64)
        for _ in range(args.warmup):
            gv.rk_step(Uv, rk, cfl=w.cfl)
        msv, profv = time_steps(gv, Uv, args.steps, rk, w.cfl, profile=True)
        line["variants"]["fp64_viscous"] = {
            "value": cells * stages * args.steps / (msv / 1e3), "unit": UNIT, "ms_per_step": msv / args.steps,
            "mu": mu, "prandtl": wv.prandtl, "reynolds": 1000,
            "stencil_ms_per_step": profv[0] / args.steps,
            "viscous_and_ghost_ms_per_step": msv / args.steps - profv[0] / args.steps,
            "note": "FP64 Navier-Stokes: edge ghosts + primitives + viscous residual kernels before each stage"}
        del gv, Uv
        if args.workload != "c4":
            line["variants"]["c4_lattice"] = lattice_variant(args, peaks, peak_src, world)
        if args.workload == "c3" and args.n is None:
            line["variants"]["c5_ramp"] = ramp_variant(args, peaks, peak_src, world)

    # the performance model of Sec. 6 on this GPU: the 2D ramp at three N_l
    # with N_w = 1024, each cut into P = 1, 4, 16, 64 i-blocks (the model's
    # 1D decomposition along N_l); fitted t_I, t_B, beta of the FP64 step
    if world == 1 and not args.no_perf_model:
        from paper_2305_18057_gb300 import perfmodel, workloads as wl
        sizes = (2048, 4096, 8192)
        rows, fit = perfmodel.decomposition_study(
            [wl.ramp_2d(ni=n, nj=1024) for n in sizes], (1, 4, 16, 64),
            lambda w_: gpu_setup(w_, sensei.FP64)[:2], steps=10, warmup=3)
        line["perf_model"] = {
            "workload": "ramp2d N_l x 1024, N_l in {2048, 4096, 8192}, cut into P in {1, 4, 16, 64} i-blocks, "
                        "FP64 SSPRK3 step",
            "fit": "T_step = N t_I + N_B t_B + t_0 (N_B = cells on block faces)",
            "t_I_ns": fit["t_I"] * 1e9, "t_B_ns": fit["t_B"] * 1e9, "t_0_us": fit["t_0"] * 1e6,
            "beta": fit["beta"], "max_rel_dev": fit["max_rel_dev"],
            "samples": [[r["dims"][0], r["parts"], r["boundary_cells"], round(r["step_s"] * 1e3, 4)]
                        for r in rows],
            "samples_cols": ["N_l", "P", "N_B", "ms_per_step"]}

    if world == 1 and not args.no_perf_model and args.workload == "c3":
        line["heterogeneous"] = hetero_study(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle_leg(args, w, line, main_prec)
    # NEXT row f4 by the model of Sec. 6 (Eq. hete with alpha = 0): adding C
    # host cores to one GPU that is r_gc times one core (the oracle, as a
    # stand-in CPU worker) shrinks the interior term by (r_gc + C) / r_gc
    if "perf_model" in line and "cpu_baseline" in line:
        one = line["cpu_baseline"]["one_core"]["value"]
        r_gc = value / one
        cores = os.cpu_count() or 1
        line["perf_model"]["heterogeneous"] = {
            "r_gc_vs_oracle_core": r_gc, "host_cores": cores,
            "cpu_share_of_cells": cores / (r_gc + cores),
            "model_speedup_vs_gpu_only": (r_gc + cores) / r_gc,
            "note": "Eq. hete, interior term, ideal overlap, with one oracle core as the CPU worker's speed"}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
