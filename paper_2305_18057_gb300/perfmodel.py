"""The paper's performance model (Sec. 6) restated, and its inputs measured
on one GB300 with this library's kernels.

Model (Sec. 6, Eqs. sequential, cpu, gpu, hete, alpha, beta): one iteration
on an N_l x N_w (x N_d) domain costs N cells x t_I for the interior plus the
boundary cells x t_B, plus transfers and synchronisations; with C CPU workers
and G GPU workers r_gc times faster than a CPU, a 1D decomposition along N_l
gives each worker N_l / (G r_gc + C) columns, and with t_f = alpha T_b and
t_B = beta t_I the time per iteration becomes

    [N_l N_w / (G r_gc + C) + (2 N_w + 2 N_l / (G r_gc + C)) (1 + alpha) beta] t_I.

The functions below are those equations as printed (Eq. cpu is labelled
time_gpu in the paper; it is the C-CPU time).  On one GPU there are no host
transfers (t_DH = t_HH = t_HD = 0), and t_I and t_B are not separable inside
one fused kernel, so `decomposition_study` measures them the way the model
uses them: it times whole steps of the same grids cut into P blocks along
N_l (every cut adds 2 N_w boundary cells) and fits T = N t_I + N_B t_B + t_0,
t_0 standing for the per-step launch and synchronisation terms (5 t_S).
"""
from __future__ import annotations


def time_seq(Nl, Nw, Nd, tI, tB, tDH=0.0, tHH=0.0, tHD=0.0, tS=0.0):
    """Eq. sequential: one iteration on one worker, 3D domain."""
    return Nl * Nw * Nd * tI + (2 * Nl * Nw + 2 * Nl * Nd + 2 * Nw * Nd) * tB + tDH + tHH + tHD + 5 * tS


def time_cpu(Nl, Nw, C, tI, tB, tDH=0.0, tHH=0.0, tHD=0.0, tS=0.0):
    """Eq. cpu: C CPU workers, 2D domain decomposed along N_l."""
    return Nl * Nw / C * tI + (2 * Nw + 2 * Nl / C) * tB + tDH + tHH + tHD + 5 * tS


def time_gpu(Nl, Nw, G, rgc, tI, tB, tDH=0.0, tHH=0.0, tHD=0.0, tS=0.0):
    """Eq. gpu: G GPU workers each r_gc times a CPU."""
    return Nl * Nw / (G * rgc) * tI + (2 * Nw + 2 * Nl / (G * rgc)) * tB + tDH + tHH + tHD + 5 * tS


def time_hete(Nl, Nw, G, rgc, C, tI, tB, tDH=0.0, tHH=0.0, tHD=0.0, tS=0.0):
    """Eq. hete: G GPUs and C CPUs sharing the columns by speed."""
    w = G * rgc + C
    return Nl * Nw / w * tI + (2 * Nw + 2 * Nl / w) * tB + tDH + tHH + tHD + 5 * tS


def time_alpha(Nl, Nw, G, rgc, C, tI, tB, alpha):
    """Eq. alpha: transfers and synchronisation folded into alpha T_b."""
    w = G * rgc + C
    return Nl * Nw / w * tI + (2 * Nw + 2 * Nl / w) * tB * (1.0 + alpha)


def time_beta(Nl, Nw, G, rgc, C, tI, alpha, beta):
    """Eq. beta: t_B = beta t_I."""
    w = G * rgc + C
    return (Nl * Nw / w + (2 * Nw + 2 * Nl / w) * (1.0 + alpha) * beta) * tI


def boundary_cells(dims):
    """Cells on the boundary faces of every block (the paper's boundary-domain
    cells: 2(N_l N_w + N_l N_d + N_w N_d) per 3D block, 2(N_l + N_w) in 2D)."""
    n = 0
    for ni, nj, nk in dims:
        n += 2 * (ni + nj) if nk == 1 else 2 * (ni * nj + ni * nk + nj * nk)
    return n


def fit(samples):
    """Least-squares t_I, t_B and a per-step constant t_0 (the 5 t_S launch
    and synchronisation term of the model) from measured step times:
    T = N t_I + N_B t_B + t_0 per step, rows weighted by 1/T so
    that every configuration counts alike.  samples: [(N, N_B, T)]."""
    import numpy as np
    A = np.array([[n, nb, 1.0] for n, nb, _ in samples], dtype=np.float64)
    T = np.array([t for _, _, t in samples], dtype=np.float64)
    w = 1.0 / T
    x, *_ = np.linalg.lstsq(A * w[:, None], T * w, rcond=None)
    pred = A @ x
    return {"t_I": float(x[0]), "t_B": float(x[1]), "t_0": float(x[2]), "beta": float(x[1] / x[0]),
            "max_rel_dev": float(np.max(np.abs(pred - T) / T))}


def decomposition_study(workloads, parts, setup, steps=10, warmup=3, rk=1):
    """The model's 1D decomposition on one GPU: every workload cut into P
    i-blocks for each P in `parts` (interfaces between the cuts), timed per
    step with CUDA events after `warmup` steps; returns the samples and the
    fitted t_I, t_B, beta.  setup(w) -> (grid, states) builds the library's
    grid for a workload."""
    import torch
    from . import workloads as wl
    rows = []
    for w in workloads:
        for P in parts:
            ws = wl.split_i(w, P) if P > 1 else w
            g, Us = setup(ws)
            for _ in range(warmup):
                g.rk_step(Us, rk, cfl=ws.cfl)
            s = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s)
            for _ in range(steps):
                g.rk_step(Us, rk, cfl=ws.cfl)
            e1.record(s)
            torch.cuda.synchronize()
            T = e0.elapsed_time(e1) / steps / 1e3
            rows.append({"dims": list(w.dims[0]), "parts": P, "cells": ws.cells,
                         "boundary_cells": boundary_cells(ws.dims), "step_s": T})
            g.close()
            del g, Us
    f = fit([(r["cells"], r["boundary_cells"], r["step_s"]) for r in rows])
    return rows, f
