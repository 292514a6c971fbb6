"""Pins of the oracle against solutions the mathematics fixes:

* Sod's shock tube against the exact Riemann solution (Toro, ch. 4), along
  i, j and k, with the error falling as the grid is refined;
* smooth advection of a density bump (an exact Euler solution): second-order
  convergence of the whole scheme;
* a manufactured steady solution on a curvilinear periodic grid: second-order
  truncation error of the spatial residual (Eq. residual with source S_h);
* a Mach-4 compression ramp: the plateau pressure and shock angle of the
  weak oblique shock (theta-beta-Mach);
* the paper's inflow table (golden fixture) turned into the freestream state.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from exact import oblique_jumps, riemann_sample, riemann_star, weak_beta
from helpers import oracle_grid, oracle_states
from paper_2305_18057_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = 1.4


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_exact_solvers_match_textbook():
    sod = _golden("sod_star.json")
    L, R = sod["left"], sod["right"]
    ps, us = riemann_star((L["rho"], L["u"], L["p"]), (R["rho"], R["u"], R["p"]), sod["gamma"])
    assert round(ps, sod["digits"]) == sod["p_star"] and round(us, sod["digits"]) == sod["u_star"]
    for case in _golden("oblique_shock.json")["cases"]:
        beta, p21, _, _ = oblique_jumps(case["mach"], math.radians(case["theta_deg"]))
        assert abs(math.degrees(beta) - case["beta_deg"]) < 0.01
        assert abs(p21 - case["p_ratio"]) < 0.005


def test_inlet_inflow_state():
    t = _golden("inlet_inflow.json")
    prim = wl.inlet_inflow(mach=t["mach"], p=t["pressure_pa"], T=t["temperature_k"])
    rho, u, v, w, p = prim
    assert abs(rho - 0.197017) < 1e-6 and abs(p - 12270.0) < 1e-9
    c = math.sqrt(G * p / rho)
    assert abs(c - 295.281) < 1e-3 and abs(u / c - 4.0) < 1e-12 and v == 0.0 and w == 0.0


def _sod(N, axis, t_end=0.2, cfl=0.4):
    ni, nj, nk = [(N, 1, 1), (1, N, 1), (2, 2, N)][axis]
    X = wl.cartesian_nodes(ni, nj, nk)
    xc = wl.cell_centres(X)[axis]
    left = xc < 0.5
    U0 = wl.conserved(np.where(left, 1.0, 0.125), 0.0, 0.0, 0.0, np.where(left, 1.0, 0.1))
    bcs = wl.bcs_all(wl.PERIODIC)
    bcs[2 * axis] = wl.BC(wl.EXTRAPOLATE)
    bcs[2 * axis + 1] = wl.BC(wl.EXTRAPOLATE)
    w = wl.Workload("sod", [(ni, nj, nk)], [X], [U0], [bcs], limiter="vanleer")
    g = oracle_grid(w)
    Us = oracle_states(g, w)
    # fixed dt from the largest wave speed of the problem (|u| + c < 2), so
    # the same steps are taken whatever the cell shape across the tube
    steps = int(math.ceil(t_end / (cfl * (1.0 / N) / 2.0)))
    for _ in range(steps):
        g.rk_step(Us, oracle.RK3_SSP, dt=t_end / steps)
    rho = np.moveaxis(g.interior(Us[0], 0)[0], 2 - axis, 0).reshape(N, -1)[:, 0]
    x = (np.arange(N) + 0.5) / N
    ex, _, _ = riemann_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / t_end)
    return float(np.mean(np.abs(rho - ex)))


def test_sod_shock_tube_converges_to_exact_solution():
    errs = [_sod(N, 0) for N in (100, 200, 400)]
    assert errs[0] > errs[1] > errs[2]
    order = math.log(errs[0] / errs[2], 4.0)
    assert order >= 0.6, (errs, order)
    assert errs[2] < 6e-3, errs


@pytest.mark.parametrize("axis", [1, 2])
def test_sod_along_j_and_k(axis):
    e = _sod(100, axis)
    assert abs(e - _sod(100, 0)) < 1e-12


def _advect(n, limiter, t_end=0.05):
    w = wl.advection_2d(n=n, seed=5)
    g = oracle_grid(w, limiter=limiter)
    Us = oracle_states(g, w)
    # constant dt scaled with h: a fixed CFL of the uniform flow
    dt = 0.4 * (1.0 / n) / (2.0 * (math.cos(math.pi / 6) + math.sin(math.pi / 6)) + 2.0)
    steps = int(round(t_end / dt))
    dt = t_end / steps
    for _ in range(steps):
        g.rk_step(Us, oracle.RK3_SSP, dt=dt)
    centre = [float(v) for v in w.note.split("[")[1].split("]")[0].split(",")]
    xc = wl.cell_centres(w.nodes[0])
    u, v = 2.0 * math.cos(math.pi / 6), 2.0 * math.sin(math.pi / 6)
    exact = 1.0 + wl.bump(xc[0] - u * t_end, xc[1] - v * t_end, centre)
    return float(np.mean(np.abs(g.interior(Us[0], 0)[0] - exact)))


@pytest.mark.parametrize("limiter,min_order", [("none", 1.9), ("vanleer", 1.6)])
def test_smooth_advection_second_order(limiter, min_order):
    e1, e2 = _advect(32, limiter), _advect(64, limiter)
    order = math.log2(e1 / e2)
    assert order >= min_order, (e1, e2, order)


def _mms_truncation(n, kappa):
    """max |R_h / |Omega| | with R_h = sum_f F.S - |Omega| S(x_c) for the
    manufactured periodic state W(x, y); S = div F(W) analytically."""
    import sympy as sp
    x, y = sp.symbols("x y")
    tp = 2 * sp.pi
    rho = 1 + sp.Rational(1, 5) * sp.sin(tp * x) * sp.cos(tp * y)
    u = 1 + sp.Rational(3, 10) * sp.cos(tp * x)
    v = sp.Rational(1, 2) + sp.Rational(1, 5) * sp.sin(tp * y)
    p = 1 + sp.Rational(1, 4) * sp.cos(tp * (x + y))
    E = p / (G - 1) + rho * (u * u + v * v) / 2
    Fx = [rho * u, rho * u * u + p, rho * u * v, 0, (E + p) * u]
    Fy = [rho * v, rho * u * v, rho * v * v + p, 0, (E + p) * v]
    S = [sp.lambdify((x, y), sp.diff(Fx[q], x) + sp.diff(Fy[q], y), "numpy") for q in range(5)]
    W = [sp.lambdify((x, y), f, "numpy") for f in (rho, u, v, p)]
    X = wl.periodic_sine_nodes(n, n, 1, amplitude_cells=3.0, seed=7)
    xc = wl.cell_centres(X)
    cx, cy = xc[0], xc[1]
    U0 = wl.conserved(W[0](cx, cy), W[1](cx, cy), W[2](cx, cy), 0.0, W[3](cx, cy))
    w = wl.Workload("mms", [(n, n, 1)], [X], [U0], [wl.bcs_all(wl.PERIODIC)], kappa=kappa)
    g = oracle_grid(w, limiter="none", kappa=kappa)
    vol = g.metrics(0)[3]
    src = np.zeros((5, 1, n, n))
    for q in range(5):
        src[q] = vol * (np.broadcast_to(S[q](cx, cy), vol.shape) if q != 3 else 0.0)
    R = g.residual(oracle_states(g, w), src=[src])[0]
    return float(np.max(np.abs(R / vol)))


@pytest.mark.parametrize("kappa", [1.0 / 3.0, -1.0])
def test_manufactured_solution_second_order(kappa):
    e = [_mms_truncation(n, kappa) for n in (16, 32, 64)]
    o1, o2 = math.log2(e[0] / e[1]), math.log2(e[1] / e[2])
    assert o2 >= 1.9, (e, o1, o2)


def test_compression_ramp_oblique_shock():
    """Mach 4 over a 10-deg ramp, run to a steady state: the pressure plateau
    on the ramp and the shock angle follow theta-beta-Mach."""
    ni, nj = 96, 48
    X = wl.ramp_nodes(ni, nj, 1, length=1.0, height=0.5, corner=0.2, angle_deg=10.0, ratio=1.0)
    prim = wl.normalized_freestream(4.0, (1.0, 0.0, 0.0))
    bcs = [wl.BC(wl.INFLOW, prim), wl.BC(wl.EXTRAPOLATE), wl.BC(wl.SLIP_WALL), wl.BC(wl.INFLOW, prim),
           wl.BC(wl.PERIODIC), wl.BC(wl.PERIODIC)]
    w = wl.Workload("ramp", [(ni, nj, 1)], [X], [wl.uniform_state((ni, nj, 1), prim)], [bcs],
                    limiter="vanleer")
    g = oracle_grid(w)
    Us = oracle_states(g, w)
    for it in range(1200):
        _, (l2, _, _) = g.rk_step(Us, oracle.RK3_SSP, cfl=0.8)
        if it == 0:
            l2_0 = l2[0]
    assert l2[0] < 1e-5 * l2_0, (l2[0], l2_0)
    beta, p21, _, _ = oblique_jumps(4.0, math.radians(10.0))
    I = g.interior(Us[0], 0)
    pfield = (G - 1.0) * (I[4] - 0.5 * (I[1] ** 2 + I[2] ** 2 + I[3] ** 2) / I[0])
    p1 = prim[4]
    xc = wl.cell_centres(X)
    # plateau: wall-adjacent cells on the ramp, away from the corner and outflow
    sel = (xc[0, 0, 0] > 0.45) & (xc[0, 0, 0] < 0.9)
    plateau = pfield[0, 0, sel].mean() / p1
    assert abs(plateau - p21) < 0.02 * p21, (plateau, p21)
    # shock angle: where p crosses the mid-jump value along vertical lines
    pm = 0.5 * (1.0 + p21) * p1
    pts = []
    for i in range(ni):
        xline = xc[0, 0, :, i]
        if xline[0] < 0.45 or xline[0] > 0.95:
            continue
        col = pfield[0, :, i]
        yl = xc[1, 0, :, i]
        above = np.nonzero(col < pm)[0]
        if above.size == 0:
            continue
        jj = above[0]
        if jj == 0:
            continue
        t = (col[jj - 1] - pm) / (col[jj - 1] - col[jj])
        pts.append((xline[jj], yl[jj - 1] + t * (yl[jj] - yl[jj - 1])))
    pts = np.array(pts)
    slope = np.polyfit(pts[:, 0], pts[:, 1], 1)[0]
    assert abs(math.degrees(math.atan(slope)) - math.degrees(beta)) < 1.0, (math.degrees(math.atan(slope)),
                                                                           math.degrees(beta))
