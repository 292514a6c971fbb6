"""Pins of the oracle's MUSCL extrapolation (Eq. flux, Sec. 5) and limiters."""
import numpy as np
import pytest

import oracle

LIMITED = [oracle.LIM_MINMOD, oracle.LIM_VANLEER]
ALL = [oracle.LIM_NONE] + LIMITED


def test_limiter_values():
    mm, vl = oracle.LIM_MINMOD, oracle.LIM_VANLEER
    assert oracle.psi(mm, -1.0) == 0.0 and oracle.psi(mm, 0.5) == 0.5 and oracle.psi(mm, 3.0) == 1.0
    assert oracle.psi(vl, -2.0) == 0.0 and oracle.psi(vl, 1.0) == 1.0
    assert abs(oracle.psi(vl, 3.0) - 1.5) < 1e-15          # (3+3)/(1+3)
    for lim in LIMITED:
        for r in (0.1, 0.7, 1.0, 2.5, 40.0):
            # symmetry psi(r)/r = psi(1/r): the property that makes kappa drop out
            assert abs(oracle.psi(lim, r) / r - oracle.psi(lim, 1.0 / r)) < 1e-15


@pytest.mark.parametrize("lim", ALL)
@pytest.mark.parametrize("kappa", [-1.0, 0.0, 1.0 / 3.0, 0.5])
def test_constant_and_linear_data_are_exact(lim, kappa):
    for q in ([2.0, 2.0, 2.0, 2.0], [0.0, 0.0, 0.0, 0.0]):
        assert oracle.muscl(q, lim, kappa) == (q[1], q[1])
    a, b = 0.7, -0.3
    q = [a + b * i for i in range(4)]           # cells i-1..i+2 at 0..3, face at 1.5
    qL, qR = oracle.muscl(q, lim, kappa)
    assert abs(qL - (a + 1.5 * b)) < 1e-15 and abs(qR - (a + 1.5 * b)) < 1e-15


def test_kappa_third_reproduces_quadratic_face_value():
    # cell averages of x^2 over unit cells centred on 0..3 are i^2 + 1/12; the
    # unlimited kappa = 1/3 scheme returns the point value (1.5)^2 at the face
    q = [i * i + 1.0 / 12.0 for i in range(4)]
    qL, qR = oracle.muscl(q, oracle.LIM_NONE, 1.0 / 3.0)
    assert abs(qL - 2.25) < 1e-14 and abs(qR - 2.25) < 1e-14
    # kappa = -1 (fully upwind) is only exact for linear data
    qL, _ = oracle.muscl(q, oracle.LIM_NONE, -1.0)
    assert abs(qL - 2.25) > 1e-3


@pytest.mark.parametrize("lim", LIMITED)
def test_tvd_bounds_and_kappa_independence(lim):
    rng = np.random.default_rng(7)
    for _ in range(20000):
        q = rng.normal(size=4) * rng.choice([1e-3, 1.0, 1e3])
        if rng.uniform() < 0.2:
            q[rng.integers(4)] = q[rng.integers(4)]   # flat differences
        qL, qR = oracle.muscl(q, lim, 1.0 / 3.0)
        lo, hi = min(q[1], q[2]), max(q[1], q[2])
        tol = 1e-14 * (abs(lo) + abs(hi))
        assert lo - tol <= qL <= hi + tol
        assert lo - tol <= qR <= hi + tol
        qL2, qR2 = oracle.muscl(q, lim, -1.0)
        assert abs(qL2 - qL) <= 4e-16 * (abs(qL) + np.abs(q).max())
        assert abs(qR2 - qR) <= 4e-16 * (abs(qR) + np.abs(q).max())


@pytest.mark.parametrize("lim", LIMITED)
def test_slope_form(lim):
    # for a symmetric limiter Eq. flux collapses to q_i + (eps/2) sigma_i with
    # sigma = minmod(dm, dp) or 2 dm dp / (dm + dp) (dm dp > 0), else 0
    rng = np.random.default_rng(8)
    for _ in range(5000):
        q = rng.normal(size=4)
        dm, d0, dp = q[1] - q[0], q[2] - q[1], q[3] - q[2]
        if lim == oracle.LIM_MINMOD:
            s1 = 0.0 if dm * d0 <= 0 else np.sign(dm) * min(abs(dm), abs(d0))
            s2 = 0.0 if d0 * dp <= 0 else np.sign(d0) * min(abs(d0), abs(dp))
        else:
            s1 = 0.0 if dm * d0 <= 0 else 2 * dm * d0 / (dm + d0)
            s2 = 0.0 if d0 * dp <= 0 else 2 * d0 * dp / (d0 + dp)
        qL, qR = oracle.muscl(q, lim, 0.2, eps=1.0)
        assert abs(qL - (q[1] + 0.5 * s1)) < 1e-14
        assert abs(qR - (q[2] - 0.5 * s2)) < 1e-14


def test_first_order_when_eps_zero():
    q = [0.0, 1.0, 5.0, -2.0]
    for lim in ALL:
        assert oracle.muscl(q, lim, 1.0 / 3.0, eps=0.0) == (1.0, 5.0)
