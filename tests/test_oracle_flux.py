"""Pins of the oracle's inviscid flux F_{i,n} (Eq. governing) and Roe flux.

Closed-form flux values, consistency, conservation (antisymmetry), Roe's
property, supersonic upwinding, the exact stationary normal shock,
rotational invariance and the entropy-fix switch."""
import math

import numpy as np
import pytest

import oracle
from exact import normal_shock_state

G = 1.4


def _rand_state(rng, mach=None):
    rho = rng.uniform(0.3, 3.0)
    p = rng.uniform(0.3, 3.0)
    c = math.sqrt(G * p / rho)
    u = rng.normal(size=3)
    if mach is not None:
        u *= mach * c / np.linalg.norm(u)
    return np.array([rho, *u, p])


def test_euler_flux_closed_form():
    # W = (rho, u, v, w, p) = (1, 2, 0, 0, 1) through n = x: mass 2, momentum
    # rho u^2 + p = 5, energy (p/(g-1) + rho u^2/2 + p) u = (2.5 + 2 + 1) 2 = 11
    np.testing.assert_allclose(oracle.euler_flux([1, 2, 0, 0, 1], [1, 0, 0]), [2, 5, 0, 0, 11], rtol=1e-15)
    # same state through the area vector (0, 2, 0): only pressure, scaled by 2
    np.testing.assert_allclose(oracle.euler_flux([1, 2, 0, 0, 1], [0, 2, 0]), [0, 0, 2, 0, 0], atol=1e-15)
    # rho = 2, (u, v, w) = (1, 1, 0), p = 3, n = (1, 1, 0)/sqrt2 with |S| = sqrt2:
    # mass 2*2, x-mom 2*1*2 + 1*3, z-mom 0, energy (7.5 + 2 + 3) * 2
    np.testing.assert_allclose(oracle.euler_flux([2, 1, 1, 0, 3], [1, 1, 0]), [4, 7, 7, 0, 25], rtol=1e-14)


def test_roe_consistency():
    rng = np.random.default_rng(1)
    for _ in range(200):
        W = _rand_state(rng)
        S = rng.normal(size=3)
        np.testing.assert_allclose(oracle.roe_flux(W, W, S), oracle.euler_flux(W, S), rtol=1e-14, atol=1e-14)


def test_roe_antisymmetry():
    rng = np.random.default_rng(2)
    for _ in range(200):
        WL, WR, S = _rand_state(rng), _rand_state(rng), rng.normal(size=3)
        a = oracle.roe_flux(WL, WR, S)
        b = oracle.roe_flux(WR, WL, -S)
        np.testing.assert_allclose(a, -b, rtol=1e-13, atol=1e-13)


def test_roe_property():
    # sum_k lam_k alpha_k r_k = F(W_R) - F(W_L) for any pair of states
    rng = np.random.default_rng(3)
    for _ in range(300):
        WL, WR, S = _rand_state(rng), _rand_state(rng), rng.normal(size=3)
        J = oracle.roe_jump(WL, WR, S)
        dF = oracle.euler_flux(WR, S) - oracle.euler_flux(WL, S)
        scale = np.abs(oracle.euler_flux(WL, S)).max() + np.abs(oracle.euler_flux(WR, S)).max()
        assert np.max(np.abs(J - dF)) < 1e-13 * scale


@pytest.mark.parametrize("fix", [0.0, 0.1])
def test_supersonic_upwinding(fix):
    rng = np.random.default_rng(4)
    n = np.array([0.6, 0.0, 0.8])
    for _ in range(100):
        WL = _rand_state(rng)
        WR = _rand_state(rng)
        # make both states supersonic along +n and close enough that the Roe
        # average is too: every wave speed positive, the fix inactive
        for W in (WL, WR):
            c = math.sqrt(G * W[4] / W[0])
            W[1:4] = 3.0 * c * n + 0.1 * rng.normal(size=3)
        F = oracle.roe_flux(WL, WR, 2.0 * n, fix=fix)
        np.testing.assert_allclose(F, oracle.euler_flux(WL, 2.0 * n), rtol=1e-12, atol=1e-12)
        # along -n every wave runs from the right state to the left one
        F = oracle.roe_flux(WR, WL, -2.0 * n, fix=fix)
        np.testing.assert_allclose(F, oracle.euler_flux(WL, -2.0 * n), rtol=1e-12, atol=1e-12)


def test_stationary_normal_shock_is_exact_without_fix():
    # Rankine-Hugoniot states of a stationary shock: Roe's linearisation
    # recognises the jump as one wave of speed 0, so F = F(W_L) = F(W_R).
    for M in (1.5, 2.0, 4.0):
        rho1, p1 = 1.2, 0.9
        u1 = M * math.sqrt(G * p1 / rho1)
        rho2, u2, p2 = normal_shock_state(rho1, u1, p1)
        WL = [rho1, u1, 0.0, 0.0, p1]
        WR = [rho2, u2, 0.0, 0.0, p2]
        F = oracle.roe_flux(WL, WR, [1, 0, 0], fix=0.0)
        FL = oracle.euler_flux(WL, [1, 0, 0])
        FR = oracle.euler_flux(WR, [1, 0, 0])
        np.testing.assert_allclose(FL, FR, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(F, FL, rtol=1e-12, atol=1e-12)
        # with Harten's fix the zero-speed wave gets dissipation: no longer exact
        Ff = oracle.roe_flux(WL, WR, [1, 0, 0], fix=0.1)
        assert np.max(np.abs(Ff - FL)) > 1e-6


def test_rotational_invariance():
    rng = np.random.default_rng(5)
    for _ in range(100):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        WL, WR, S = _rand_state(rng), _rand_state(rng), rng.normal(size=3)
        rot = lambda W: np.array([W[0], *(Q @ W[1:4]), W[4]])
        a = oracle.roe_flux(WL, WR, S)
        b = oracle.roe_flux(rot(WL), rot(WR), Q @ S)
        np.testing.assert_allclose(rot(a), b, rtol=1e-12, atol=1e-12)


def test_entropy_fix_only_below_delta_and_continuous():
    # transonic pair: the Roe-averaged V_n - a crosses 0 as the left speed varies
    WR = np.array([1.0, 1.0, 0.0, 0.0, 1.0 / G])
    a = 1.0
    for uL in np.linspace(0.6, 1.4, 41):
        WL = np.array([1.0, uL, 0.0, 0.0, 1.0 / G])
        f0 = oracle.roe_flux(WL, WR, [1, 0, 0], fix=0.0)
        f1 = oracle.roe_flux(WL, WR, [1, 0, 0], fix=0.1)
        lam = 0.5 * (uL + 1.0) - a   # equal densities: Roe average is the arithmetic mean
        if abs(lam) > 0.1 * a * 1.05:
            np.testing.assert_allclose(f0, f1, rtol=0, atol=1e-14)
    # continuity across |lam| = delta
    eps = 1e-9
    for s in (-1, 1):
        target = 0.1 * s
        f = []
        for d in (-eps, eps):
            uL = 2 * (1.0 + target + d) - 1.0
            # keep the sound speed of the Roe average at 1 by fixing H
            WL = np.array([1.0, uL, 0.0, 0.0, 1.0 / G])
            f.append(oracle.roe_flux(WL, WR, [1, 0, 0], fix=0.1))
        assert np.max(np.abs(f[0] - f[1])) < 1e-6
