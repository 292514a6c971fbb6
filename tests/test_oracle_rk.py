"""Pins of the oracle's explicit Runge-Kutta (Eq. runge_kutta).

* the tableaux satisfy the order conditions and have the stability
  polynomials of the Shu-Osher forms of SSPRK(2,2), SSPRK(3,3), SSPRK(4,2);
* one full step of the Euler solver on a density wave advected through a
  periodic box (where the discrete operator is linear) multiplies each
  Fourier mode by P(dt * lambda), lambda the exact symbol of the unlimited
  MUSCL-kappa upwind operator;
* a uniform state with a constant source S is integrated exactly,
  U^{n+1} = U^n + dt S (with the 1/|Omega| of Eq. spatial_residual)."""
import numpy as np
import pytest

import oracle
from helpers import oracle_grid, oracle_states
from paper_2305_18057_gb300 import workloads as wl

# stability polynomial coefficients (1, z, z^2, ...) of the Shu-Osher forms:
# SSPRK(2,2): 1/2 + 1/2 (1+z)^2;  SSPRK(3,3): 1 + z + z^2/2 + z^3/6;
# SSPRK(4,2): 1/4 + 3/4 (1 + z/3)^4
POLY = {
    oracle.RK2_SSP: [1.0, 1.0, 0.5],
    oracle.RK3_SSP: [1.0, 1.0, 0.5, 1.0 / 6.0],
    oracle.RK4_SSP2: [1.0, 1.0, 0.5, 1.0 / 9.0, 1.0 / 108.0],
}


def _stability_poly(a, b, z):
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * a, np.ones(s))


@pytest.mark.parametrize("rk", list(POLY))
def test_tableau_order_and_stability_polynomial(rk):
    a, b = oracle.rk_tableau(rk)
    c = a.sum(axis=1)
    assert np.allclose(np.triu(a), 0.0)              # explicit: a_ij = 0 for i <= j
    assert abs(b.sum() - 1.0) < 1e-15 and abs(b @ c - 0.5) < 1e-15
    if rk == oracle.RK3_SSP:
        assert abs(b @ c ** 2 - 1 / 3) < 1e-15 and abs(b @ a @ c - 1 / 6) < 1e-15
    for z in (-0.3, -1.0 + 0.5j, -2.0, 0.7j):
        want = sum(cf * z ** k for k, cf in enumerate(POLY[rk]))
        assert abs(_stability_poly(a, b, z) - want) < 1e-14


@pytest.mark.parametrize("rk", list(POLY))
@pytest.mark.parametrize("kappa", [1.0 / 3.0, -1.0, 0.0])
def test_full_step_amplifies_fourier_modes_by_stability_polynomial(rk, kappa):
    N, Uvel, m = 32, 1.7, 3
    X = wl.cartesian_nodes(N, 1, 1, lengths=(1.0, 0.25, 1.0))
    xc = wl.cell_centres(X)[0].ravel()
    eps_amp = 1e-3
    rho = 1.0 + eps_amp * np.cos(2 * np.pi * m * xc + 0.4)
    U0 = wl.conserved(rho.reshape(1, 1, N), Uvel, 0.0, 0.0, 1.0)
    w = wl.Workload("wave", [(N, 1, 1)], [X], [U0], [wl.bcs_all(wl.PERIODIC)], kappa=kappa)
    g = oracle_grid(w, limiter="none", kappa=kappa)
    Us = oracle_states(g, w)
    h = 1.0 / N
    dt = 0.4 * h / Uvel
    g.rk_step(Us, rk, dt=dt)
    rho1 = g.interior(Us[0], 0)[0, 0, 0]
    th = 2 * np.pi * m / N
    # face value rho^L_{i+1/2} = rho_i (1 + (1/4)[(1-k)(1-e^{-i th}) + (1+k)(e^{i th}-1)])
    gfac = 1.0 + 0.25 * ((1 - kappa) * (1 - np.exp(-1j * th)) + (1 + kappa) * (np.exp(1j * th) - 1))
    lam = -(Uvel / h) * (1 - np.exp(-1j * th)) * gfac
    P = sum(cf * (dt * lam) ** k for k, cf in enumerate(POLY[rk]))
    c0 = np.fft.fft(rho - 1.0)[m]
    c1 = np.fft.fft(rho1 - 1.0)[m]
    assert abs(c1 - P * c0) < 1e-10 * abs(c0)
    # the mean is conserved and the other modes stay empty
    spec = np.abs(np.fft.fft(rho1 - 1.0))
    spec[[m, N - m]] = 0.0
    assert spec.max() < 1e-10 * abs(c0)


@pytest.mark.parametrize("rk", list(POLY))
def test_constant_source_integrates_exactly(rk):
    n = 4
    X = wl.cartesian_nodes(n, n, n, lengths=(0.5, 0.7, 0.9))
    prim = (1.2, 0.3, -0.2, 0.5, 0.8)
    w = wl.Workload("src", [(n, n, n)], [X], [wl.uniform_state((n, n, n), prim)], [wl.bcs_all(wl.PERIODIC)])
    g = oracle_grid(w)
    Us = oracle_states(g, w)
    Sdens = np.array([0.1, -0.2, 0.3, 0.05, 0.7])
    vol = g.metrics(0)[3]
    src = np.ascontiguousarray(Sdens[:, None, None, None] * vol[None])
    U_before = g.interior(Us[0], 0).copy()
    dt = 1e-2
    g.rk_step(Us, rk, dt=dt, src=[src])
    got = g.interior(Us[0], 0)
    np.testing.assert_allclose(got, U_before + dt * Sdens[:, None, None, None], rtol=1e-13, atol=1e-15)
