"""sensei_rk_steps and its graph: nsteps steps in one call give the results
of nsteps sensei_rk_step calls bit for bit (states, each step's dt, the
recorded norms).  In the 3D FP32-storage form the last Runge-Kutta stage of
each step forms the next step's CFL bound from the state it writes, with the
time-step reduction's FP32 rule (the same device function), and the next
step skips the reduction: the bits must not move, and the reduction must run
only once per call."""
import numpy as np
import pytest

from helpers import gpu_grid, gpu_states
from paper_2305_18057_gb300 import sensei, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "periodic3d": lambda: wl.periodic_3d(n=40, nj=24, nk=20, seed=5),
    "lattice": lambda: wl.lattice_3d(sizes=(6, 9, 13), nblk=(2, 2, 2), seed=4, perturb=0.05),
    "ramp3d": lambda: wl.ramp_3d(ni=48, nj=32, nk=16, perturb=0.05),
    "ramp2d": lambda: wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05),
}
PRECISIONS = {"fp64": sensei.FP64, "fp32_flux": sensei.FP32_FLUX, "fp32_store": sensei.FP32_STORE}
NSTEPS = 6


def _run(w, precision, how):
    g = gpu_grid(w, precision=precision)
    Us = gpu_states(g, w)
    dts = torch.zeros(NSTEPS, dtype=torch.float64, device=Us[0].device)
    g.profile(True)
    g.profile_read(reset=True)
    if how == "single":
        for n in range(NSTEPS):
            g.rk_step(Us, sensei.RK3_SSP, cfl=0.5, dt_used=dts[n:n + 1])
    elif how == "multi":
        g.rk_steps(Us, NSTEPS, sensei.RK3_SSP, cfl=0.5, dt_used=dts)
    else:
        g.profile(False)
        graph = g.steps_graph(Us, NSTEPS, sensei.RK3_SSP, cfl=0.5, dt_used=dts)
        graph.launch()
        graph.close()
    torch.cuda.synchronize()
    launches = g.profile_read(reset=True)[2]
    g.profile(False)
    _, l2, linf, cons = g.norms()
    states = [g.download(U, b) for b, U in enumerate(Us)]
    return states, dts.cpu().numpy(), np.concatenate([l2, linf, cons]), launches


@pytest.mark.parametrize("precision", sorted(PRECISIONS))
@pytest.mark.parametrize("case", sorted(CASES))
def test_rk_steps_equal_single_steps_bitwise(case, precision):
    w = CASES[case]()
    prec = PRECISIONS[precision]
    s1, dt1, n1, k1 = _run(w, prec, "single")
    s2, dt2, n2, k2 = _run(w, prec, "multi")
    assert np.array_equal(dt1, dt2), (dt1, dt2)
    assert np.all(dt1 > 0) and len(set(dt1.tolist())) > 1   # the state moves, so dt does
    for a, b in zip(s1, s2):
        assert np.array_equal(a, b)
    assert np.array_equal(n1, n2)
    # the time-step reduction runs once per call where the bound is fused
    fused = prec == sensei.FP32_STORE and all(d[2] > 1 for d in w.dims)
    assert k1 - k2 == (NSTEPS - 1 if fused else 0), (k1, k2)


@pytest.mark.parametrize("precision", ["fp32_flux", "fp32_store"])
def test_steps_graph_equals_rk_steps_bitwise(precision):
    w = CASES["lattice"]()
    s1, dt1, n1, _ = _run(w, PRECISIONS[precision], "multi")
    s2, dt2, n2, _ = _run(w, PRECISIONS[precision], "graph")
    assert np.array_equal(dt1, dt2)
    for a, b in zip(s1, s2):
        assert np.array_equal(a, b)
    assert np.array_equal(n1, n2)


@pytest.mark.parametrize("rk", [sensei.RK2_SSP, sensei.RK4_SSP2])
def test_rk_steps_other_schemes_and_a_given_dt(rk):
    """The fused bound in two- and four-stage schemes (its last stage is the
    second or the fourth), and a given dt (no bound at all), both bitwise."""
    w = CASES["periodic3d"]()
    for cfl, dt in ((0.5, 0.0), (0.0, 2e-4)):
        out = []
        for how in ("single", "multi"):
            g = gpu_grid(w, precision=sensei.FP32_STORE)
            Us = gpu_states(g, w)
            if how == "single":
                for _ in range(4):
                    g.rk_step(Us, rk, cfl=cfl, dt=dt)
            else:
                g.rk_steps(Us, 4, rk, cfl=cfl, dt=dt)
            torch.cuda.synchronize()
            out.append(g.download(Us[0], 0))
        assert np.array_equal(out[0], out[1]), (rk, cfl)


def test_rk_steps_rejects_no_steps():
    w = CASES["periodic3d"]()
    g = gpu_grid(w, precision=sensei.FP32_FLUX)
    Us = gpu_states(g, w)
    with pytest.raises(Exception):
        g.rk_steps(Us, 0, sensei.RK3_SSP, cfl=0.5)
