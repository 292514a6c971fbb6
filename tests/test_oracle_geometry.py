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


def _trilinear_volume_exact(X, i, j, k):
    """Volume of cell (i, j, k) as the integral of det J of the trilinear map
    of its 8 nodes over the unit cube, in exact rational arithmetic: det J
    has degree <= 2 in each variable, so Simpson's rule (nodes 0, 1/2, 1)
    in each direction is exact."""
    from fractions import Fraction as F
    c = {(a, b, d): [F(float(X[q, k + d, j + b, i + a])) for q in range(3)]
         for a in (0, 1) for b in (0, 1) for d in (0, 1)}
    nodes, wts = (F(0), F(1, 2), F(1)), (F(1, 6), F(4, 6), F(1, 6))
    total = F(0)
    for s, ws in zip(nodes, wts):
        for t, wt in zip(nodes, wts):
            for u, wu in zip(nodes, wts):
                lin = lambda z, e: z if e else 1 - z
                J = [[F(0)] * 3 for _ in range(3)]
                for (a, b, d), x in c.items():
                    g = (lin(t, b) * lin(u, d) * (1 if a else -1),
                         lin(s, a) * lin(u, d) * (1 if b else -1),
                         lin(s, a) * lin(t, b) * (1 if d else -1))
                    for q in range(3):
                        for r in range(3):
                            J[q][r] += x[q] * g[r]
                det = (J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
                       - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
                       + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]))
                total += ws * wt * wu * det
    return total


def test_thin_curved_cells_far_from_the_origin_keep_their_volume():
    """Cells 1e-6 thin in j, 3 units from the coordinate origin, with twisted
    (non-planar) faces: the oracle's volume against the exact volume of the
    trilinear cell through the same (double) nodes.  The volume is measured
    from each cell's corner, so it keeps full relative accuracy; measured
    from the coordinate origin its terms ~|x| h^2 would cancel to h^3 and lose
    ~|x|/h (about 1e-9 relative here)."""
    ni, nj, nk = 3, 2, 2
    rng = np.random.default_rng(11)
    xi = np.stack(np.meshgrid(np.arange(nk + 1) / nk, np.arange(nj + 1) / nj, np.arange(ni + 1) / ni,
                              indexing="ij")[::-1])    # (3, nk+1, nj+1, ni+1): xi_i, xi_j, xi_k
    A = np.array([[0.7, 0.0, 0.05], [0.0, 1e-6, 0.0], [0.03, 0.0, 0.45]])
    X = np.einsum("ab,bkji->akji", A, xi) + np.array([3.1, 2.7, -2.9])[:, None, None, None]
    X[1] += 1e-7 * rng.uniform(-1.0, 1.0, size=X[1].shape)   # twist the thin faces
    X = np.ascontiguousarray(X)
    vol = _grid(X, ni, nj, nk).metrics(0)[3]
    for k in range(nk):
        for j in range(nj):
            for i in range(ni):
                exact = float(_trilinear_volume_exact(X, i, j, k))
                assert exact > 0
                assert abs(vol[k, j, i] - exact) <= 1e-13 * exact, (i, j, k, vol[k, j, i], exact)
