"""The host worker of heterogeneous co-execution (Sec. 4: the host cores'
share of a step) against the oracle, on the CPU: the residual of Eq.
residual to 1e-12 of each variable's scale, the CFL time step to 1e-14,
and SSPRK steps (Eq. runge_kutta) to 1e-11, with every boundary rule it
takes and each limiter; host threads change no result."""
import numpy as np
import pytest

import oracle
from helpers import oracle_grid, oracle_states, per_var_rel
from paper_2305_18057_gb300 import build as libbuild
from paper_2305_18057_gb300 import workloads as wl


@pytest.fixture(scope="module")
def sensei():
    libbuild.build()
    from paper_2305_18057_gb300 import sensei as s
    s.load()
    return s


def _host(sensei, w, limiter=None, threads=1, recon_conserved=False):
    ni, nj, nk = w.dims[0]
    h = sensei.HostBlock(w.dims[0], w.nodes[0], gamma=w.gamma, limiter=wl.LIMITERS[limiter or w.limiter],
                         kappa=w.kappa, eps=w.eps, entropy_fix=w.fix, reconstruct_conserved=recon_conserved,
                         threads=threads)
    for f, bc in enumerate(w.bcs[0]):
        h.set_bc(f, bc.type, bc.prim)
    h.interior()[...] = w.U0[0]
    return h


CASES = {
    "periodic": lambda: wl.periodic_3d(n=22, nj=17, nk=13, seed=31),
    "ramp": lambda: wl.ramp_3d(ni=20, nj=14, nk=9, perturb=0.05, seed=32),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("limiter", ["none", "minmod", "vanleer"])
def test_host_residual_matches_oracle(sensei, case, limiter):
    w = CASES[case]()
    h = _host(sensei, w, limiter)
    og = oracle_grid(w, limiter=limiter)
    Uo = oracle_states(og, w)
    Ro = og.residual(Uo)[0]
    R = h.residual()
    assert per_var_rel(R, Ro) < 1e-12


def test_host_conserved_reconstruction(sensei):
    w = CASES["ramp"]()
    h = _host(sensei, w, recon_conserved=True)
    og = oracle_grid(w, recon_conserved=True)
    Uo = oracle_states(og, w)
    assert per_var_rel(h.residual(), og.residual(Uo)[0]) < 1e-12


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_steps_match_oracle(sensei, case):
    w = CASES[case]()
    h = _host(sensei, w)
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    for rk, orc in ((sensei.RK3_SSP, oracle.RK3_SSP), (sensei.RK2_SSP, oracle.RK2_SSP),
                    (sensei.RK4_SSP2, oracle.RK4_SSP2)):
        for _ in range(3):
            dt = h.dt_min(0.5)
            dt_o = 0.5 * og.dt_min(Uo)
            assert abs(dt - dt_o) <= 1e-14 * dt_o
            h.step(rk, dt)
            og.rk_step(Uo, orc, dt=dt)
    assert per_var_rel(h.interior(), og.interior(Uo[0], 0)) < 1e-11


def test_host_threads_bitwise(sensei):
    w = CASES["periodic"]()
    a = _host(sensei, w, threads=1)
    b = _host(sensei, w, threads=3)
    for h in (a, b):
        for _ in range(2):
            h.step(sensei.RK3_SSP, h.dt_min(0.5))
    np.testing.assert_array_equal(a.interior(), b.interior())


def test_host_rejects_unsupported(sensei):
    w = CASES["periodic"]()
    with pytest.raises(sensei.SenseiError):
        sensei.HostBlock((1, 4, 4), w.nodes[0][:, :5, :5, :2])
