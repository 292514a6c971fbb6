"""The double-float form (SENSEI_DF64: reconstruction and Roe flux in pairs
of FP32 numbers, about 48 significant bits, on an FP64 state) against the
FP64 oracle on the small parity cases, where it meets the FP64 path's own
tolerances: one residual 1e-11 relative per variable, the state after 100
steps 1e-9.  (On fine grids, where the residual is a small difference of
large fluxes, its 32x larger unit roundoff shows: the full-size test holds
it to 32 times the FP64 bar.)"""
import numpy as np
import pytest

import oracle
from helpers import gpu_grid, gpu_states, oracle_grid, oracle_states, per_var_rel
from paper_2305_18057_gb300 import sensei, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "periodic3d_odd": lambda: wl.periodic_3d(n=37, nj=19, nk=11, seed=3),
    "ramp3d": lambda: wl.ramp_3d(ni=40, nj=20, nk=9, ratio=1.05, perturb=0.05),
    "advection2d": lambda: wl.advection_2d(n=48),
    "ramp2d": lambda: wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05),
    "lattice": lambda: wl.lattice_3d(sizes=(6, 9, 13), nblk=(2, 2, 2), seed=4, perturb=0.05),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("limiter", ["none", "minmod", "vanleer"])
def test_df64_residual_parity(case, limiter):
    w = CASES[case]()
    og = oracle_grid(w, limiter=limiter)
    Ro = og.residual(oracle_states(og, w))
    g = gpu_grid(w, limiter=limiter, precision=sensei.DF64)
    Us = gpu_states(g, w)
    Rs = [torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device) for ni, nj, nk in w.dims]
    g.residual(Us, Rs)
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(Rs[b].cpu().numpy(), Ro[b]) < 1e-11, (case, limiter, b)


@pytest.mark.parametrize("case", ["periodic3d_odd", "ramp2d", "lattice"])
def test_df64_state_after_100_steps(case):
    w = CASES[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w, precision=sensei.DF64)
    Us = gpu_states(g, w)
    dt_used = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    for _ in range(100):
        g.rk_step(Us, sensei.RK3_SSP, cfl=0.5, dt_used=dt_used)
        og.rk_step(Uo, oracle.RK3_SSP, dt=dt_used.item())
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(g.download(Us[b], b), og.interior(Uo[b], b)) < 1e-9, (case, b)


def test_df64_with_viscosity():
    w = wl.periodic_3d(n=37, nj=19, nk=11, seed=3)
    rng = np.random.default_rng(21)
    U = w.U0[0].copy()
    U[1:4] *= 1.0 + 0.05 * rng.uniform(-1.0, 1.0, size=U[1:4].shape)
    w.U0 = [U]
    w.mu = 0.02
    og = oracle_grid(w)
    Ro = og.residual(oracle_states(og, w))
    g = gpu_grid(w, precision=sensei.DF64)
    Us = gpu_states(g, w)
    Rs = [torch.empty((5, 11, 19, 37), dtype=torch.float64, device=Us[0].device)]
    g.residual(Us, Rs)
    torch.cuda.synchronize()
    assert per_var_rel(Rs[0].cpu().numpy(), Ro[0]) < 1e-11


def test_df64_step_graph_replays_eager_steps_bitwise():
    w = CASES["lattice"]()
    ga = gpu_grid(w, precision=sensei.DF64)
    Ua = gpu_states(ga, w)
    gb = gpu_grid(w, precision=sensei.DF64)
    Ub = gpu_states(gb, w)
    graph = gb.step_graph(Ub, oracle.RK3_SSP, cfl=0.5)
    for _ in range(5):
        ga.rk_step(Ua, oracle.RK3_SSP, cfl=0.5)
        graph.launch()
    torch.cuda.synchronize()
    graph.close()
    for b in range(len(w.dims)):
        assert torch.equal(ga.interior_view(Ua[b], b), gb.interior_view(Ub[b], b)), b


@pytest.mark.parametrize("case", ["periodic3d_odd", "ramp2d", "lattice"])
def test_df64_local_time_stepping_and_autotune(case):
    """Local time stepping and the autotuned schedule in the double-float
    form, 20 steps against the oracle at the FP64 path's 1e-9."""
    w = CASES[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w, precision=sensei.DF64)
    Us = gpu_states(g, w)
    g.autotune(Us)
    dt_min = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    for _ in range(20):
        g.rk_step_local(Us, oracle.RK3_SSP, cfl=0.6, dt_min=dt_min)
        dto, _ = og.rk_step_local(Uo, oracle.RK3_SSP, cfl=0.6)
        assert abs(dt_min.item() - dto) <= 1e-11 * dto
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(g.download(Us[b], b), og.interior(Uo[b], b)) < 1e-9, (case, b)
