"""Mixed precision against the FP64 oracle: FP32 reconstruction and flux on
an FP64 state (FP32_FLUX), and additionally FP32 stage storage with the FP64
accumulation U^{n+1} = U^n + D (FP32_STORE).  No closed form fixes this
error, so it is measured and bounded.  Target: density L2 error <= 1e-5
relative to the oracle after many steps; each residual within FP32
rounding of the flux; conservation sums still FP64-exact."""
import numpy as np
import pytest

from helpers import gpu_grid, gpu_states, oracle_grid, oracle_states, per_var_rel
from paper_2305_18057_gb300 import sensei, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _l2_rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["periodic3d", "ramp2d", "lattice"])
def test_fp32_flux_residual_close_to_oracle(case):
    w = {"periodic3d": lambda: wl.periodic_3d(n=37, nj=19, nk=11, seed=3),
         "ramp2d": lambda: wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05),
         "lattice": lambda: wl.lattice_3d(sizes=(6, 9, 13), nblk=(2, 2, 2), seed=4, perturb=0.05)}[case]()
    og = oracle_grid(w)
    Ro = og.residual(oracle_states(og, w))
    g = gpu_grid(w, precision=sensei.FP32_FLUX)
    Us = gpu_states(g, w)
    Rs = [torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device) for ni, nj, nk in w.dims]
    g.residual(Us, Rs)
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        # a flux difference of FP32 fluxes: absolute error ~ 1e-7 of the flux
        # scale, which for these perturbed fields is ~1e-5 of max |R|
        assert per_var_rel(Rs[b].cpu().numpy(), Ro[b]) < 2e-4, (case, b)


@pytest.mark.parametrize("precision", ["fp32_flux", "fp32_store"])
@pytest.mark.parametrize("case,steps", [("periodic3d", 100), ("ramp2d", 100), ("advection2d", 100),
                                        ("lattice", 60)])
def test_mixed_state_error_within_target(case, steps, precision):
    w = {"periodic3d": lambda: wl.periodic_3d(n=24, nj=16, nk=12, seed=8),
         "ramp2d": lambda: wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05),
         "advection2d": lambda: wl.advection_2d(n=48),
         "lattice": lambda: wl.lattice_3d(sizes=(6, 9, 13), nblk=(2, 2, 2), seed=4, perturb=0.05)}[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w, precision={"fp32_flux": sensei.FP32_FLUX, "fp32_store": sensei.FP32_STORE}[precision])
    Us = gpu_states(g, w)
    dt_used = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    for _ in range(steps):
        g.rk_step(Us, sensei.RK3_SSP, cfl=0.5, dt_used=dt_used)
        og.rk_step(Uo, 1, dt=dt_used.item())
    torch.cuda.synchronize()
    got = np.concatenate([g.download(Us[b], b).reshape(5, -1) for b in range(len(w.dims))], axis=1)
    want = np.concatenate([og.interior(Uo[b], b).reshape(5, -1) for b in range(len(w.dims))], axis=1)
    err_rho = _l2_rel(got[0], want[0])
    assert err_rho <= 1e-5, err_rho
    # momentum and energy: same order
    for q in (1, 2, 4):
        assert _l2_rel(got[q], want[q]) <= 1e-4, q


@pytest.mark.parametrize("precision", ["fp32_flux", "fp32_store"])
def test_mixed_conserves_mass_to_round_off(precision):
    w = wl.periodic_3d(n=24, nj=16, nk=12, seed=8)
    g = gpu_grid(w, precision={"fp32_flux": sensei.FP32_FLUX, "fp32_store": sensei.FP32_STORE}[precision])
    Us = gpu_states(g, w)
    g.rk_step(Us, sensei.RK3_SSP, cfl=0.5)
    st, _, _, cons0 = g.norms()
    for _ in range(50):
        g.rk_step(Us, sensei.RK3_SSP, cfl=0.5)
    st, _, _, cons1 = g.norms()
    # each FP32 face flux enters its two cells with opposite signs; the
    # per-cell FP32 sums and (FP32_STORE) the FP32 increments round, so the
    # FP64 sums of |Omega| U drift only at the level of FP32 rounding of
    # the per-step change, far below the FP32 rounding of the state itself
    tol = 1e-12 if precision == "fp32_flux" else 1e-10
    assert abs(cons1[0] - cons0[0]) <= tol * abs(cons0[0])
    assert abs(cons1[4] - cons0[4]) <= tol * abs(cons0[4])


@pytest.mark.parametrize("precision", ["fp32_flux", "fp32_store", "df64"])
@pytest.mark.parametrize("rk", ["rk2", "rk4"])
def test_every_runge_kutta_scheme_in_every_form(precision, rk):
    """SSPRK(2,2) and SSPRK(4,2) (the RK3 cases are above) in the FP32 forms
    (the FP32-storage increments carry each scheme's own coefficients) and the
    double-float form, 40 steps against the oracle stepped with the GPU's dt:
    density L2 1e-5 for the FP32 forms, 1e-9 per variable for double-float."""
    import oracle
    prec = {"fp32_flux": sensei.FP32_FLUX, "fp32_store": sensei.FP32_STORE, "df64": sensei.DF64}[precision]
    rkg = {"rk2": sensei.RK2_SSP, "rk4": sensei.RK4_SSP2}[rk]
    rko = {"rk2": oracle.RK2_SSP, "rk4": oracle.RK4_SSP2}[rk]
    for w in (wl.periodic_3d(n=24, nj=16, nk=12, seed=8), wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05)):
        og = oracle_grid(w)
        Uo = oracle_states(og, w)
        g = gpu_grid(w, precision=prec)
        Us = gpu_states(g, w)
        dt_used = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
        for _ in range(40):
            g.rk_step(Us, rkg, cfl=0.5, dt_used=dt_used)
            og.rk_step(Uo, rko, dt=dt_used.item())
        torch.cuda.synchronize()
        got, want = g.download(Us[0], 0), og.interior(Uo[0], 0)
        if precision == "df64":
            assert per_var_rel(got, want) < 1e-9, (w.name, rk)
        else:
            assert _l2_rel(got[0], want[0]) <= 1e-5, (w.name, rk)


@pytest.mark.parametrize("precision", ["fp32_flux", "fp32_store"])
@pytest.mark.parametrize("case", ["periodic3d", "lattice"])
def test_mixed_local_time_stepping_within_target(case, precision):
    """Local time steps (each cell its own CFL step) in the FP32 forms: the
    3D FP32 stencil's local-step instantiations against the oracle's local
    steps, at the mixed forms' state bar."""
    w = {"periodic3d": lambda: wl.periodic_3d(n=24, nj=16, nk=12, seed=8),
         "lattice": lambda: wl.lattice_3d(sizes=(6, 9, 13), nblk=(2, 2, 2), seed=4, perturb=0.05)}[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w, precision={"fp32_flux": sensei.FP32_FLUX, "fp32_store": sensei.FP32_STORE}[precision])
    Us = gpu_states(g, w)
    for _ in range(30):
        g.rk_step_local(Us, sensei.RK3_SSP, cfl=0.6)
        og.rk_step_local(Uo, 1, cfl=0.6)
    torch.cuda.synchronize()
    got = np.concatenate([g.download(Us[b], b).reshape(5, -1) for b in range(len(w.dims))], axis=1)
    want = np.concatenate([og.interior(Uo[b], b).reshape(5, -1) for b in range(len(w.dims))], axis=1)
    moved = _l2_rel(np.concatenate([og.interior(oracle_states(og, w)[b], b).reshape(5, -1)
                                    for b in range(len(w.dims))], axis=1)[0], want[0])
    assert moved > 1e-4, moved
    assert _l2_rel(got[0], want[0]) <= 1e-5
