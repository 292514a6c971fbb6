"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle,
element by element, on seeded inputs spanning several tiles and ragged tails.

Tolerances: one residual 1e-11 relative (per variable, scaled by the largest
oracle value of that variable); the state after 100 steps 1e-9; dt 1e-14;
the conservation sums 1e-13."""
import numpy as np
import pytest

import oracle
from helpers import gpu_grid, gpu_states, oracle_grid, oracle_states, per_var_rel
from paper_2305_18057_gb300 import sensei, workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RK = {"rk2": 0, "rk3": 1, "rk4": 2}

CASES = {
    # i: 37 = 32 + 5 (ragged i tile), j: 19 = 8 + 8 + 3, k: 11
    "periodic3d_odd": lambda: wl.periodic_3d(n=37, nj=19, nk=11, seed=3),
    # inflow, extrapolation, slip wall on the ramp, periodic k
    "ramp3d": lambda: wl.ramp_3d(ni=40, nj=20, nk=9, ratio=1.05, perturb=0.05),
    "advection2d": lambda: wl.advection_2d(n=48),
    "ramp2d": lambda: wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05),
    # 8 uneven blocks, interface ghost exchange in every direction
    "lattice": lambda: wl.lattice_3d(sizes=(6, 9, 13), nblk=(2, 2, 2), seed=4, perturb=0.05),
}


def _residuals(w, limiter=None, kappa=None, recon=False, fix=None, precision=0):
    og = oracle_grid(w, limiter=limiter, kappa=kappa, recon_conserved=recon, fix=fix)
    Ro = og.residual(oracle_states(og, w))
    g = gpu_grid(w, limiter=limiter, kappa=kappa, recon_conserved=recon, fix=fix, precision=precision)
    Us = gpu_states(g, w)
    Rs = [torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device) for ni, nj, nk in w.dims]
    g.residual(Us, Rs)
    torch.cuda.synchronize()
    return [R.cpu().numpy() for R in Rs], Ro, g, og, Us


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("limiter", ["none", "minmod", "vanleer"])
def test_residual_parity(case, limiter):
    w = CASES[case]()
    Rg, Ro, *_ = _residuals(w, limiter=limiter)
    for b in range(len(w.dims)):
        assert per_var_rel(Rg[b], Ro[b]) < 1e-11, (case, limiter, b)


@pytest.mark.parametrize("case", ["periodic3d_odd", "ramp2d"])
def test_residual_parity_options(case):
    w = CASES[case]()
    for kw in (dict(limiter="none", kappa=-1.0), dict(limiter="minmod", recon=True), dict(limiter="vanleer", fix=0.0),
               dict(limiter="vanleer", fix=0.3, recon=True)):
        Rg, Ro, *_ = _residuals(w, **kw)
        assert per_var_rel(Rg[0], Ro[0]) < 1e-11, kw


@pytest.mark.parametrize("precision,tol", [(sensei.DF64, 1e-11), (sensei.FP32_FLUX, 2e-4), (sensei.FP32_STORE, 2e-4)])
def test_residual_options_in_every_precision_form(precision, tol):
    """The unlimited kappa form, conserved reconstruction and the entropy fix
    off or wider, in the double-float form (at the FP64 bar) and the FP32
    forms (at their residual bar, FP32 rounding of the fluxes)."""
    for case in ("periodic3d_odd", "ramp2d"):
        w = CASES[case]()
        for kw in (dict(limiter="none", kappa=-1.0), dict(limiter="minmod", recon=True),
                   dict(limiter="vanleer", fix=0.0), dict(limiter="vanleer", fix=0.3, recon=True)):
            Rg, Ro, *_ = _residuals(w, precision=precision, **kw)
            assert per_var_rel(Rg[0], Ro[0]) < tol, (case, kw)


@pytest.mark.parametrize("precision,tol", [(sensei.DF64, 1e-11), (sensei.FP32_FLUX, 2e-4), (sensei.FP32_STORE, 2e-4)])
def test_residual_with_source_and_norms_in_every_precision_form(precision, tol):
    """The source term, the residual norms and the conservation sums in the
    double-float and FP32 forms (the norms of the FP32 residual, the
    conservation sums FP64 in every form)."""
    w = CASES["periodic3d_odd"]()
    ni, nj, nk = w.dims[0]
    rng = np.random.default_rng(0)
    src = rng.normal(size=(5, nk, nj, ni)) * 1e-4
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    Ro = og.residual(Uo, src=[np.ascontiguousarray(src)])
    g = gpu_grid(w, precision=precision)
    Us = gpu_states(g, w)
    R = torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device)
    g.residual(Us, [R], [torch.as_tensor(src, device=R.device)])
    st, l2, linf, cons = g.norms()
    assert per_var_rel(R.cpu().numpy(), Ro[0]) < tol
    ol2, olinf, ocons = og.norms(Ro, Uo)
    np.testing.assert_allclose(l2, ol2, rtol=10 * tol)
    np.testing.assert_allclose(linf, olinf, rtol=10 * tol)
    np.testing.assert_allclose(cons, ocons, rtol=1e-13, atol=1e-13 * np.abs(ocons).max())


def test_residual_with_source_and_norms():
    w = CASES["periodic3d_odd"]()
    ni, nj, nk = w.dims[0]
    rng = np.random.default_rng(0)
    src = rng.normal(size=(5, nk, nj, ni)) * 1e-4
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    Ro = og.residual(Uo, src=[np.ascontiguousarray(src)])
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    R = torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device)
    g.residual(Us, [R], [torch.as_tensor(src, device=R.device)])
    st, l2, linf, cons = g.norms()
    assert per_var_rel(R.cpu().numpy(), Ro[0]) < 1e-11
    ol2, olinf, ocons = og.norms(Ro, Uo)
    np.testing.assert_allclose(l2, ol2, rtol=1e-11)
    np.testing.assert_allclose(linf, olinf, rtol=1e-11)
    np.testing.assert_allclose(cons, ocons, rtol=1e-13, atol=1e-13 * np.abs(ocons).max())


@pytest.mark.parametrize("case", list(CASES))
def test_dt_parity(case):
    w = CASES[case]()
    og = oracle_grid(w)
    dto = 0.5 * og.dt_min(oracle_states(og, w))
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    dt_used = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    g.rk_step(Us, RK["rk3"], cfl=0.5, dt_used=dt_used)
    assert abs(dt_used.item() - dto) <= 1e-14 * dto


@pytest.mark.parametrize("case,rk,steps", [("periodic3d_small", "rk3", 100), ("advection2d", "rk3", 100),
                                           ("ramp2d", "rk2", 100), ("lattice", "rk4", 100),
                                           ("ramp3d", "rk3", 30)])
def test_state_after_many_steps(case, rk, steps):
    w = wl.periodic_3d(n=24, nj=16, nk=12, seed=8) if case == "periodic3d_small" else CASES[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    dt_used = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    for n in range(steps):
        g.rk_step(Us, RK[rk], cfl=0.5, dt_used=dt_used)
        # same dt on both sides: the oracle takes the GPU's dt explicitly
        # (dt itself is checked by test_dt_parity)
        og.rk_step(Uo, RK[rk], dt=dt_used.item())
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(g.download(Us[b], b), og.interior(Uo[b], b)) < 1e-9, (case, b)


def test_norms_of_step_match_oracle():
    w = CASES["ramp3d"]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    g.rk_step(Us, RK["rk3"], dt=1e-7)
    st, l2, linf, cons = g.norms()
    _, (ol2, olinf, ocons) = og.rk_step(Uo, RK["rk3"], dt=1e-7)
    np.testing.assert_allclose(l2, ol2, rtol=1e-11)
    np.testing.assert_allclose(linf, olinf, rtol=1e-11)
    np.testing.assert_allclose(cons, ocons, rtol=1e-13)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_nonphysical_state_is_reported(precision):
    w = CASES["periodic3d_odd"]()
    U0 = [w.U0[0].copy()]
    U0[0][4, 3, 5, 7] = 0.0          # rho e_t = 0: negative pressure in one cell
    g = gpu_grid(w, precision=precision)
    Us = gpu_states(g, w, U0)
    g.rk_step(Us, RK["rk3"], dt=1e-6)
    st, *_ = g.norms(check=False)
    assert st == sensei.ERR_NONPHYSICAL
    # the flag is cleared once reported
    g.upload(Us[0], 0, w.U0[0])
    g.rk_step(Us, RK["rk3"], dt=1e-6)
    st, *_ = g.norms(check=False)
    assert st == sensei.OK


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_step_graph_replays_eager_steps_bitwise(precision):
    # a CUDA graph of one step (ghost fill, dt, three persistent stencil
    # launches, norm finalisation) replayed on the lattice gives exactly the
    # eagerly launched steps
    w = CASES["lattice"]()
    ga = gpu_grid(w, precision=precision)
    Ua = gpu_states(ga, w)
    gb = gpu_grid(w, precision=precision)
    Ub = gpu_states(gb, w)
    graph = gb.step_graph(Ub, RK["rk3"], cfl=0.5)
    for _ in range(5):
        ga.rk_step(Ua, RK["rk3"], cfl=0.5)
        graph.launch()
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert torch.equal(ga.interior_view(Ua[b], b), gb.interior_view(Ub[b], b)), b
    graph.close()


@pytest.mark.parametrize("case", ["periodic3d_odd", "lattice"])
def test_autotuned_schedule_keeps_parity(case):
    w = CASES[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    kchunk, persistent = g.autotune(Us)
    assert kchunk in (4, 8, 16, 32, 64, 128)
    # the autotuner's dt = 0 launches leave the interior untouched
    for b in range(len(w.dims)):
        np.testing.assert_array_equal(g.download(Us[b], b), w.U0[b])
    dt_used = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    for _ in range(20):
        g.rk_step(Us, RK["rk3"], cfl=0.5, dt_used=dt_used)
        og.rk_step(Uo, RK["rk3"], dt=dt_used.item())
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(g.download(Us[b], b), og.interior(Uo[b], b)) < 1e-9, b


@pytest.mark.parametrize("case", ["periodic3d_odd", "ramp2d", "lattice"])
def test_local_time_stepping_parity(case):
    w = CASES[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    dt_min = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    for _ in range(20):
        g.rk_step_local(Us, RK["rk3"], cfl=0.6, dt_min=dt_min)
        dto, _ = og.rk_step_local(Uo, RK["rk3"], cfl=0.6)
        assert abs(dt_min.item() - dto) <= 1e-11 * dto
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(g.download(Us[b], b), og.interior(Uo[b], b)) < 1e-9, (case, b)


def test_local_time_stepping_converges_on_gpu():
    # the stretched Mach-4 ramp of the oracle's pin, marched to round-off
    from test_oracle_lts import _ramp
    w = _ramp()
    for prec in (0, 1, 2, 3):
        g = gpu_grid(w, precision=prec)
        Us = gpu_states(g, w)
        g.rk_step_local(Us, RK["rk3"], cfl=0.8)
        l2_0 = g.norms()[1][0]
        for _ in range(1500):
            g.rk_step_local(Us, RK["rk3"], cfl=0.8)
        l2 = g.norms()[1][0]
        # FP64 reaches round-off, the double-float form nearly (48 bits); the
        # FP32-flux forms stall at their own rounding level
        assert l2 < {0: 1e-9, 3: 1e-8}.get(prec, 1e-4) * l2_0, (prec, l2 / l2_0)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_item_order_changes_no_result(precision):
    """Work items by descending cost (the order the autotuner may choose for
    uneven blocks) give bitwise the block-major results, norms included."""
    from paper_2305_18057_gb300 import sensei
    w = CASES["lattice"]()
    runs = []
    for order in (0, 1):
        g = gpu_grid(w, precision=precision)
        Us = gpu_states(g, w)
        g.debug_set(sensei.DEBUG_ITEM_ORDER, order)
        for _ in range(5):
            g.rk_step(Us, RK["rk3"], cfl=0.5)
        _, l2, linf, cons = g.norms()
        assert g.schedule()["order_by_cost"] == bool(order)
        runs.append(([g.download(U, b) for b, U in enumerate(Us)], l2, linf, cons))
    for a, b in zip(runs[0][0], runs[1][0]):
        np.testing.assert_array_equal(a, b)
    for x, y in zip(runs[0][1:], runs[1][1:]):
        np.testing.assert_array_equal(x, y)
