"""Pins of the oracle's residual R_h (Eq. residual), ghost cells, time step
and norms: freestream preservation on curvilinear grids, discrete
conservation, wall and boundary invariants, multiblock = single block,
axis symmetry, the closed-form time step and special-case norms."""
import math

import numpy as np
import pytest

import oracle
from helpers import oracle_grid, oracle_states
from paper_2305_18057_gb300 import workloads as wl

G = 1.4


def _uniform_workload(dims, nodes, prim, bcs):
    return wl.Workload("t", [dims], [nodes], [wl.uniform_state(dims, prim)], [bcs])


@pytest.mark.parametrize("lim", ["none", "minmod", "vanleer"])
def test_freestream_preservation_curvilinear_3d(lim):
    n = 14
    X = wl.periodic_sine_nodes(n, n, n, amplitude_cells=0.4, seed=11)
    prim = wl.normalized_freestream(2.5, (0.3, -0.5, 0.8))
    w = _uniform_workload((n, n, n), X, prim, wl.bcs_all(wl.PERIODIC))
    g = oracle_grid(w, limiter=lim)
    Us = oracle_states(g, w)
    R = g.residual(Us)[0]
    Finf = np.abs(oracle.euler_flux(prim, [1, 0, 0])).max()
    Smax = np.abs(g.metrics(0)[0]).max()
    assert np.max(np.abs(R)) / (Finf * Smax) < 1e-13


def test_freestream_preservation_2d_ramp_with_walls():
    # flow parallel to a flat wall, inflow at imin and jmax, outflow at imax:
    # on the flat part (angle 0) R vanishes to round-off everywhere
    ni, nj = 16, 8
    X = wl.ramp_nodes(ni, nj, 1, angle_deg=0.0, ratio=1.1)
    prim = wl.inlet_inflow()
    bcs = [wl.BC(wl.INFLOW, prim), wl.BC(wl.EXTRAPOLATE), wl.BC(wl.SLIP_WALL), wl.BC(wl.INFLOW, prim),
           wl.BC(wl.PERIODIC), wl.BC(wl.PERIODIC)]
    w = _uniform_workload((ni, nj, 1), X, prim, bcs)
    g = oracle_grid(w)
    R = g.residual(oracle_states(g, w))[0]
    Finf = np.abs(oracle.euler_flux(prim, [1, 0, 0])).max()
    assert np.max(np.abs(R)) / (Finf * 1.0 / nj) < 1e-13


def test_discrete_conservation_periodic():
    w = wl.periodic_3d(n=12, seed=3)
    g = oracle_grid(w)
    Us = oracle_states(g, w)
    R = g.residual(Us)[0]
    # every interior face enters two cells with opposite signs
    scale = np.abs(R).sum(axis=(1, 2, 3))
    assert np.all(np.abs(R.sum(axis=(1, 2, 3))) < 1e-14 * scale)
    cons0 = g.norms([R], Us)[2]
    for _ in range(10):
        g.rk_step(Us, oracle.RK3_SSP, cfl=0.8)
    R = g.residual(Us)[0]
    cons = g.norms([R], Us)[2]
    for q in (0, 4):
        assert abs(cons[q] - cons0[q]) < 1e-13 * abs(cons0[q])
    for q in (1, 2, 3):
        assert abs(cons[q] - cons0[q]) < 1e-13 * (abs(cons0[0]) * 2.5)


def test_multiblock_equals_single_block_bitwise():
    w = wl.lattice_3d(sizes=(3, 4, 5), nblk=(2, 2, 2), seed=1, steps=1)
    # non-uniform initial data so that every interface matters
    rng = np.random.default_rng(0)
    NI = sum(w.dims[a][0] for a in range(2))
    NJ = sum(w.dims[2 * b][1] for b in range(2))
    NK = sum(w.dims[4 * c][2] for c in range(2))
    prim = wl.inlet_inflow(mach=3.0)
    Ug = wl.uniform_state((NI, NJ, NK), prim)
    Ug *= 1.0 + 0.05 * rng.uniform(size=Ug.shape)
    io = [0, w.dims[0][0], NI]
    jo = [0, w.dims[0][1], NJ]
    ko = [0, w.dims[0][2], NK]
    Xg = np.empty((3, NK + 1, NJ + 1, NI + 1))
    U0 = []
    for b, X in enumerate(w.nodes):
        a_, b_, c_ = b % 2, (b // 2) % 2, b // 4
        Xg[:, ko[c_]:ko[c_ + 1] + 1, jo[b_]:jo[b_ + 1] + 1, io[a_]:io[a_ + 1] + 1] = X
        U0.append(np.ascontiguousarray(Ug[:, ko[c_]:ko[c_ + 1], jo[b_]:jo[b_ + 1], io[a_]:io[a_ + 1]]))
    w.U0 = U0
    gm = oracle_grid(w)
    Um = oracle_states(gm, w)
    bcs1 = [wl.BC(wl.INFLOW, prim), wl.BC(wl.EXTRAPOLATE), wl.BC(wl.SLIP_WALL), wl.BC(wl.INFLOW, prim),
            wl.BC(wl.PERIODIC), wl.BC(wl.PERIODIC)]
    w1 = wl.Workload("g", [(NI, NJ, NK)], [Xg], [Ug], [bcs1])
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


def _shock_tube_states(N, axis):
    """Sod's problem along one index direction: 2D (one cell across) along i
    or j, a 3D column (2 x 2 cells across) along k."""
    ni, nj, nk = [(N, 1, 1), (1, N, 1), (2, 2, N)][axis]
    lengths = [1.0, 1.0, 1.0]
    X = wl.cartesian_nodes(ni, nj, nk, lengths=lengths)
    xc = wl.cell_centres(X)[axis]
    left = xc < 0.5
    vel = [0.0, 0.0, 0.0]
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    U0 = wl.conserved(rho, *vel, p)
    bcs = wl.bcs_all(wl.PERIODIC)
    bcs[2 * axis] = wl.BC(wl.EXTRAPOLATE)
    bcs[2 * axis + 1] = wl.BC(wl.EXTRAPOLATE)
    return wl.Workload("sod", [(ni, nj, nk)], [X], [U0], [bcs], limiter="minmod")


def test_axis_symmetry_of_shock_tube():
    res = []
    for axis in (0, 1, 2):
        w = _shock_tube_states(40, axis)
        g = oracle_grid(w)
        Us = oracle_states(g, w)
        for _ in range(5):
            g.rk_step(Us, oracle.RK3_SSP, dt=2e-3)
        I = g.interior(Us[0], 0)
        rho = np.moveaxis(I[0], 2 - axis, 0).reshape(40, -1)[:, 0]
        mom = np.moveaxis(I[1 + axis], 2 - axis, 0).reshape(40, -1)[:, 0]
        res.append((rho, mom))
    for rho, mom in res[1:]:
        np.testing.assert_allclose(rho, res[0][0], rtol=1e-14)
        np.testing.assert_allclose(mom, res[0][1], rtol=1e-13, atol=1e-15)


def test_time_step_closed_form():
    # uniform state on a Cartesian grid: dt = CFL h / (|u| + |v| + |w| + 3c)
    n, h = 6, 1.0 / 6
    X = wl.cartesian_nodes(n, n, n)
    prim = (1.3, 0.4, -0.7, 0.2, 0.9)
    w = _uniform_workload((n, n, n), X, prim, wl.bcs_all(wl.PERIODIC))
    g = oracle_grid(w)
    c = math.sqrt(G * prim[4] / prim[0])
    expect = h / (0.4 + 0.7 + 0.2 + 3 * c)
    assert abs(g.dt_min(oracle_states(g, w)) - expect) < 1e-15 * expect * 4
    # 2D: two directions only
    X2 = wl.cartesian_nodes(n, n, 1)
    w2 = _uniform_workload((n, n, 1), X2, prim, wl.bcs_all(wl.PERIODIC))
    g2 = oracle_grid(w2)
    expect2 = h / (0.4 + 0.7 + 2 * c)
    assert abs(g2.dt_min(oracle_states(g2, w2)) - expect2) < 1e-15 * expect2 * 4


def test_ghost_cells():
    ni, nj, nk = 5, 4, 3
    X = wl.periodic_sine_nodes(ni, nj, nk, amplitude_cells=0.3, seed=2)
    rng = np.random.default_rng(4)
    U0 = wl.conserved(rng.uniform(1, 2, (nk, nj, ni)), rng.normal(size=(nk, nj, ni)),
                      rng.normal(size=(nk, nj, ni)), rng.normal(size=(nk, nj, ni)), rng.uniform(1, 2, (nk, nj, ni)))
    prim = (1.1, 0.5, 0.1, 0.2, 0.8)
    bcs = [wl.BC(wl.SLIP_WALL), wl.BC(wl.INFLOW, prim), wl.BC(wl.EXTRAPOLATE), wl.BC(wl.EXTRAPOLATE),
           wl.BC(wl.PERIODIC), wl.BC(wl.PERIODIC)]
    w = wl.Workload("bc", [(ni, nj, nk)], [X], [U0], [bcs])
    g = oracle_grid(w)
    U = oracle_states(g, w)[0]
    g.fill_ghosts([U])
    Si = g.metrics(0)[0]
    # slip wall at imin: ghost -g mirrors interior g-1; rho, rho e_t equal,
    # tangential momentum equal, normal momentum reversed
    for gl in (1, 2):
        gh = U[:, 2:2 + nk, 2:2 + nj, 2 - gl]
        ins = U[:, 2:2 + nk, 2:2 + nj, 2 + gl - 1]
        n = Si[:, :, :, 0] / np.linalg.norm(Si[:, :, :, 0], axis=0)
        assert np.array_equal(gh[0], ins[0]) and np.array_equal(gh[4], ins[4])
        mn_g = np.einsum("akj,akj->kj", gh[1:4], n)
        mn_i = np.einsum("akj,akj->kj", ins[1:4], n)
        np.testing.assert_allclose(mn_g, -mn_i, atol=1e-14)
        np.testing.assert_allclose(gh[1:4] - mn_g * n, ins[1:4] - mn_i * n, atol=1e-14)
    # inflow at imax: the freestream conserved state
    Qinf = oracle.prim_to_cons(prim)
    for gl in (1, 2):
        np.testing.assert_allclose(U[:, 2:2 + nk, 2:2 + nj, 1 + ni + gl], Qinf[:, None, None] * np.ones((1, nk, nj)))
    # extrapolation at jmin/jmax: copies of the boundary cell
    for gl in (1, 2):
        assert np.array_equal(U[:, 2:2 + nk, 2 - gl, 2:2 + ni], U[:, 2:2 + nk, 2, 2:2 + ni])
        assert np.array_equal(U[:, 2:2 + nk, 1 + nj + gl, 2:2 + ni], U[:, 2:2 + nk, 1 + nj, 2:2 + ni])
    # periodic in k
    for gl in (1, 2):
        assert np.array_equal(U[:, 2 - gl, 2:2 + nj, 2:2 + ni], U[:, 2 + nk - gl, 2:2 + nj, 2:2 + ni])
        assert np.array_equal(U[:, 1 + nk + gl, 2:2 + nj, 2:2 + ni], U[:, 2 + gl - 1, 2:2 + nj, 2:2 + ni])


def test_norms_special_cases():
    n = 4
    X = wl.cartesian_nodes(n, n, n, lengths=(2.0, 2.0, 2.0))
    w = _uniform_workload((n, n, n), X, (1.0, 0.0, 0.0, 0.0, 1.0), wl.bcs_all(wl.PERIODIC))
    g = oracle_grid(w)
    Us = oracle_states(g, w)
    R = np.zeros((5, n, n, n))
    R[2, 1, 2, 3] = -3.0              # a single nonzero entry r: L2 = |r|/sqrt(N)
    R[4] = 0.5                        # a constant: L2 = Linf = |c|
    l2, linf, cons = g.norms([R], Us)
    assert abs(l2[2] - 3.0 / 8.0) < 1e-15 and linf[2] == 3.0
    assert abs(l2[4] - 0.5) < 1e-15 and linf[4] == 0.5
    assert l2[0] == 0.0 and linf[0] == 0.0
    # sum |Omega| U over a domain of volume 8 with rho = 1, rho e_t = 2.5
    assert abs(cons[0] - 8.0) < 1e-13 and abs(cons[4] - 8.0 * 2.5) < 1e-12
