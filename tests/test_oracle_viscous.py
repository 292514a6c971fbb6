"""Pins of the oracle's viscous flux F_nu (Eq. governing with Stokes's
hypothesis, constant mu, heat conductivity mu c_p / Pr): exact discrete
values for fields the face gradients reproduce exactly, freestream and
conservation with viscosity, multiblock = single block with the block-edge
ghosts, and the decay of a viscous shear wave."""
import math

import numpy as np
import pytest

import oracle
from helpers import oracle_grid, oracle_states
from paper_2305_18057_gb300 import workloads as wl

GAMMA = 1.4


def _affine_grid(n, A, origin=(0.1, -0.2, 0.3)):
    """n^3 cells of the image of the unit cube under x = A xi + origin (a
    uniform sheared, rotated and stretched parallelepiped grid)."""
    X = wl.cartesian_nodes(n, n, n)
    Y = np.einsum("ab,bkji->akji", np.asarray(A, float), X)
    for a in range(3):
        Y[a] += origin[a]
    return np.ascontiguousarray(Y)


A_SHEAR = [[1.0, 0.3, -0.1], [0.2, 0.9, 0.15], [-0.05, 0.1, 1.1]]


def _residual_difference(X, U, mu, prandtl=0.72):
    """R(mu) - R(0) of a single block with extrapolation at every face."""
    n = X.shape[1] - 1
    w = wl.Workload("aff", [(n, n, n)], [X], [U], [wl.bcs_all(wl.EXTRAPOLATE)], limiter="minmod",
                    mu=mu, prandtl=prandtl)
    w0 = wl.Workload("aff", [(n, n, n)], [X], [U], [wl.bcs_all(wl.EXTRAPOLATE)], limiter="minmod")
    gv, g0 = oracle_grid(w), oracle_grid(w0)
    Rv = gv.residual(oracle_states(gv, w))[0]
    R0 = g0.residual(oracle_states(g0, w0))[0]
    vol = g0.metrics(0)[3]
    return Rv - R0, vol


def test_linear_velocity_gives_exact_dissipation():
    # u = G x: the stresses are constant, so the viscous momentum residual
    # vanishes and the energy residual is -|Omega| tau : G (the work of the
    # viscous stresses), exactly for the central face gradients on a uniform
    # parallelepiped grid, away from the extrapolated boundary layers
    n, mu = 10, 0.07
    X = _affine_grid(n, A_SHEAR)
    xc = wl.cell_centres(X)
    G = np.array([[0.3, -0.5, 0.2], [0.4, 0.1, -0.3], [-0.2, 0.25, -0.15]])
    vel = [sum(G[a, b] * xc[b] for b in range(3)) for a in range(3)]
    U = wl.conserved(np.ones_like(xc[0]), vel[0], vel[1], vel[2], np.full_like(xc[0], 2.0))
    dR, vol = _residual_difference(X, U, mu)
    tau = mu * (G + G.T) - 2.0 / 3.0 * mu * np.trace(G) * np.eye(3)
    phi = float(np.sum(tau * G))
    inner = (slice(None), slice(2, n - 2), slice(2, n - 2), slice(2, n - 2))
    d = dR[inner]
    v = vol[inner[1:]]
    scale = abs(phi) * v.max()
    assert np.abs(d[0]).max() == 0.0
    assert np.abs(d[1:4]).max() < 1e-14   # rounding of O(0.02) face fluxes
    np.testing.assert_allclose(d[4], -v * phi, rtol=1e-9, atol=1e-12 * scale)


def test_quadratic_temperature_gives_exact_conduction():
    # u = 0, rho = 1, p / rho quadratic: the face gradients of a quadratic
    # are exact at the face centres of a uniform parallelepiped grid, so the
    # energy residual is -k' |Omega| Laplacian(p / rho) with
    # k' = mu gamma / ((gamma - 1) Pr)
    n, mu, pr = 10, 0.05, 0.7
    X = _affine_grid(n, A_SHEAR)
    xc = wl.cell_centres(X)
    a, b, c, dxy = 0.3, -0.2, 0.45, 0.25
    p = 3.0 + a * xc[0] ** 2 + b * xc[1] ** 2 + c * xc[2] ** 2 + dxy * xc[0] * xc[1]
    zero = np.zeros_like(p)
    U = wl.conserved(np.ones_like(p), zero, zero, zero, p)
    dR, vol = _residual_difference(X, U, mu, prandtl=pr)
    kp = mu * GAMMA / ((GAMMA - 1.0) * pr)
    lap = 2.0 * (a + b + c)
    inner = (slice(None), slice(2, n - 2), slice(2, n - 2), slice(2, n - 2))
    d = dR[inner]
    v = vol[inner[1:]]
    assert np.abs(d[:4]).max() == 0.0
    np.testing.assert_allclose(d[4], -kp * v * lap, rtol=1e-9)


def test_viscous_freestream_preservation_and_conservation():
    w = wl.periodic_3d(n=10, nj=8, nk=6, seed=5)
    w.mu = 0.02
    # uniform state: zero gradients, the viscous flux vanishes exactly
    U1 = [np.broadcast_to(w.U0[0][:, :1, :1, :1], w.U0[0].shape).copy()]
    g = oracle_grid(w)
    Us = oracle_states(g, w, U0=U1)
    R = g.residual(Us)[0]
    w0 = wl.periodic_3d(n=10, nj=8, nk=6, seed=5)
    g0 = oracle_grid(w0)
    R0 = g0.residual(oracle_states(g0, w0, U0=U1))[0]
    assert np.array_equal(R, R0)
    # perturbed state on the periodic map (the map's rho/p modes are
    # isothermal at uniform velocity, so perturb the momenta too): every
    # face flux enters two cells with opposite signs, so the residual sums
    # to zero
    rng = np.random.default_rng(11)
    Up = w.U0[0].copy()
    Up[1:4] *= 1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=Up[1:4].shape)
    Us = oracle_states(g, w, U0=[Up])
    R = g.residual(Us)[0]
    Rvis_only = R - g0.residual(oracle_states(g0, w0, U0=[Up]))[0]
    assert np.abs(Rvis_only).max() > 1e-6
    for q in range(5):
        assert abs(R[q].sum()) < 1e-13 * np.abs(R[q]).sum() + 1e-300


def test_viscous_multiblock_equals_single_block_bitwise():
    # the 2x2x2 lattice against one block of the same global grid: the
    # viscous face gradients read block-edge ghosts, which the interfaces
    # must reproduce exactly
    w = wl.lattice_3d(sizes=(3, 4, 5), nblk=(2, 2, 2), seed=1, steps=1)
    rng = np.random.default_rng(0)
    NI = sum(w.dims[a][0] for a in range(2))
    NJ = sum(w.dims[2 * b][1] for b in range(2))
    NK = sum(w.dims[4 * c][2] for c in range(2))
    prim = wl.inlet_inflow(mach=3.0)
    Ug = wl.uniform_state((NI, NJ, NK), prim)
    Ug *= 1.0 + 0.05 * rng.uniform(size=Ug.shape)
    io, jo, ko = [0, w.dims[0][0], NI], [0, w.dims[0][1], NJ], [0, w.dims[0][2], NK]
    Xg = np.empty((3, NK + 1, NJ + 1, NI + 1))
    U0 = []
    for b, X in enumerate(w.nodes):
        a_, b_, c_ = b % 2, (b // 2) % 2, b // 4
        Xg[:, ko[c_]:ko[c_ + 1] + 1, jo[b_]:jo[b_ + 1] + 1, io[a_]:io[a_ + 1] + 1] = X
        U0.append(np.ascontiguousarray(Ug[:, ko[c_]:ko[c_ + 1], jo[b_]:jo[b_ + 1], io[a_]:io[a_ + 1]]))
    w.U0 = U0
    w.mu = 2e-3
    gm = oracle_grid(w)
    Um = oracle_states(gm, w)
    bcs1 = [wl.BC(wl.INFLOW, prim), wl.BC(wl.EXTRAPOLATE), wl.BC(wl.SLIP_WALL), wl.BC(wl.INFLOW, prim),
            wl.BC(wl.PERIODIC), wl.BC(wl.PERIODIC)]
    w1 = wl.Workload("g", [(NI, NJ, NK)], [Xg], [Ug], [bcs1], mu=2e-3)
    g1 = oracle_grid(w1)
    U1 = oracle_states(g1, w1)
    for _ in range(2):
        gm.rk_step(Um, oracle.RK3_SSP, dt=1e-6)
        g1.rk_step(U1, oracle.RK3_SSP, dt=1e-6)
    glob = g1.interior(U1[0], 0)
    for b in range(8):
        a_, b_, c_ = b % 2, (b // 2) % 2, b // 4
        part = glob[:, ko[c_]:ko[c_ + 1], jo[b_]:jo[b_ + 1], io[a_]:io[a_ + 1]]
        assert np.array_equal(gm.interior(Um[b], b), part)


def test_viscous_split_ramp2d_is_exact():
    # walls, inflow and outflow meet the cut interfaces at block edges
    w = wl.ramp_2d(ni=48, nj=20, perturb=0.02)
    w.mu = 1e-3
    ws = wl.split_i(w, 4)
    g1, g2 = oracle_grid(w), oracle_grid(ws)
    U1, U2 = oracle_states(g1, w), oracle_states(g2, ws)
    R1 = g1.residual(U1)[0]
    R2 = np.concatenate(g2.residual(U2), axis=3)
    assert np.array_equal(R1, R2)


def test_viscous_time_step_closed_form():
    # uniform state at rest on a Cartesian grid: dt = |Omega| / sum_d (c |S_d|
    # + 4 max(4/3, gamma) mu / (Pr rho) |S_d|^2 / |Omega|)
    n, L = 8, 2.0
    X = wl.cartesian_nodes(n, n, n, lengths=(L, L, L))
    rho, p, mu, pr = 1.3, 0.9, 0.04, 0.72
    U0 = wl.uniform_state((n, n, n), (rho, 0.0, 0.0, 0.0, p))
    w = wl.Workload("u", [(n, n, n)], [X], [U0], [wl.bcs_all(wl.PERIODIC)], mu=mu, prandtl=pr)
    g = oracle_grid(w)
    h = L / n
    S, vol = h * h, h ** 3
    c = math.sqrt(GAMMA * p / rho)
    want = vol / (3.0 * (c * S + 4.0 * max(4.0 / 3.0, GAMMA) * mu / (pr * rho) * S * S / vol))
    assert g.dt_min(oracle_states(g, w)) == pytest.approx(want, rel=1e-14)


def _shear_wave_amplitude(n, mu, t_end):
    X = wl.cartesian_nodes(n, n, 1)
    xc = wl.cell_centres(X)
    A = 0.01
    u = A * np.sin(2.0 * np.pi * xc[1])
    U0 = wl.conserved(np.ones_like(u), u, np.zeros_like(u), np.zeros_like(u), np.full_like(u, 1.0 / GAMMA))
    w = wl.Workload("shear", [(n, n, 1)], [X], [U0], [wl.bcs_all(wl.PERIODIC)], limiter="vanleer", mu=mu)
    g = oracle_grid(w)
    Us = oracle_states(g, w)
    t = 0.0
    while t < t_end - 1e-15:
        dt = min(0.5 * g.dt_min(Us), t_end - t)
        g.rk_step(Us, oracle.RK3_SSP, dt=dt)
        t += dt
    mom = g.interior(Us[0], 0)[1, 0]
    s = np.sin(2.0 * np.pi * xc[1][0])
    return float((mom * s).sum() / (s * s).sum()) / A


def test_viscous_shear_wave_decays_at_the_exact_rate():
    # u = A sin(2 pi y) with uniform rho and p is a solution of the
    # momentum equation rho du/dt = mu d2u/dy2 (up to O(A^2) viscous
    # heating): the amplitude decays like exp(-4 pi^2 mu t / rho)
    mu, t_end = 0.01, 0.4
    exact = math.exp(-4.0 * math.pi ** 2 * mu * t_end)
    e16 = abs(_shear_wave_amplitude(16, mu, t_end) - exact)
    e32 = abs(_shear_wave_amplitude(32, mu, t_end) - exact)
    assert e32 < 2e-3
    assert e16 / e32 > 3.0   # second order in space
