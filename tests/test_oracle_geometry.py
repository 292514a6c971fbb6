"""Pins of the oracle's face area vectors and cell volumes (Delta s, n and
|Omega| of Eq. residual): exact Cartesian values, closure of every cell,
the exact volume of a periodic map, the 2D shoelace area, rotation."""
import numpy as np

import oracle
from paper_2305_18057_gb300 import workloads as wl


def _grid(X, ni, nj, nk):
    return oracle.OracleGrid([(ni, nj, nk)], [X])


def test_cartesian_metrics_exact():
    ni, nj, nk = 5, 4, 3
    L = (1.5, 0.8, 0.6)
    X = wl.cartesian_nodes(ni, nj, nk, lengths=L)
    g = _grid(X, ni, nj, nk)
    Si, Sj, Sk, vol = g.metrics(0)
    hx, hy, hz = L[0] / ni, L[1] / nj, L[2] / nk
    np.testing.assert_allclose(Si[0], hy * hz, rtol=1e-14)
    np.testing.assert_allclose(Sj[1], hx * hz, rtol=1e-14)
    np.testing.assert_allclose(Sk[2], hx * hy, rtol=1e-14)
    for S, a in ((Si, (1, 2)), (Sj, (0, 2)), (Sk, (0, 1))):
        for c in a:
            assert np.max(np.abs(S[c])) < 1e-16
    np.testing.assert_allclose(vol, hx * hy * hz, rtol=1e-13)


def _closure(Si, Sj, Sk):
    """sum over the 6 faces of the outward area vector, per cell"""
    return (Si[:, :, :, 1:] - Si[:, :, :, :-1] + Sj[:, :, 1:, :] - Sj[:, :, :-1, :]
            + Sk[:, 1:, :, :] - Sk[:, :-1, :, :])


def test_cells_are_closed_on_curvilinear_grid():
    n = 12
    X = wl.periodic_sine_nodes(n, n, n, amplitude_cells=0.3, seed=5)
    g = _grid(X, n, n, n)
    Si, Sj, Sk, vol = g.metrics(0)
    s = _closure(Si, Sj, Sk)
    scale = np.max(np.abs(Si))
    assert np.max(np.abs(s)) < 1e-15 * scale * 8


def test_periodic_map_total_volume_is_one():
    # x = xi + periodic displacement maps the unit cube onto a region of volume
    # exactly 1 (det(I + grad f) integrates to 1 for periodic f), and the
    # discrete volumes telescope to the boundary faces.
    n = 10
    X = wl.periodic_sine_nodes(n, n, n, amplitude_cells=0.6, seed=3)
    g = _grid(X, n, n, n)
    vol = g.metrics(0)[3]
    assert abs(vol.sum() - 1.0) < 1e-13
    assert vol.min() > 0


def test_2d_area_equals_shoelace_and_z_components_vanish():
    ni, nj = 7, 5
    X = wl.ramp_nodes(ni, nj, 1, ratio=1.2, angle_deg=15.0)
    g = _grid(X, ni, nj, 1)
    Si, Sj, Sk, vol = g.metrics(0)
    assert np.all(Si[2] == 0.0) and np.all(Sj[2] == 0.0)
    x, y = X[0, 0], X[1, 0]
    for j in range(nj):
        for i in range(ni):
            px = [x[j, i], x[j, i + 1], x[j + 1, i + 1], x[j + 1, i]]
            py = [y[j, i], y[j, i + 1], y[j + 1, i + 1], y[j + 1, i]]
            area = 0.5 * sum(px[m] * py[(m + 1) % 4] - px[(m + 1) % 4] * py[m] for m in range(4))
            assert abs(vol[0, j, i] - area) < 1e-14 * abs(area) * 10
    # i-face of a 2D cell: (dy, -dx, 0) times the unit depth
    for j in range(nj):
        dx = x[j + 1, 0] - x[j, 0]
        dy = y[j + 1, 0] - y[j, 0]
        np.testing.assert_allclose(Si[:2, 0, j, 0], [dy, -dx], rtol=1e-14, atol=1e-16)


def test_metrics_rotate_with_the_grid():
    n = 4
    X = wl.periodic_sine_nodes(n, n, n, amplitude_cells=0.4, seed=9)
    rng = np.random.default_rng(0)
    Qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] *= -1
    Xr = np.einsum("ab,bkji->akji", Qm, X) + np.array([0.3, -1.0, 2.0])[:, None, None, None]
    a = _grid(X, n, n, n).metrics(0)
    b = _grid(np.ascontiguousarray(Xr), n, n, n).metrics(0)
    for Sa, Sb in zip(a[:3], b[:3]):
        np.testing.assert_allclose(np.einsum("ab,b...->a...", Qm, Sa), Sb, atol=1e-15)
    np.testing.assert_allclose(a[3], b[3], rtol=1e-12)
