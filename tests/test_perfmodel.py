"""The performance model of Sec. 6 as restated in perfmodel.py: the
equations reduce to each other as the paper derives them."""
import pytest

from paper_2305_18057_gb300 import perfmodel as pm


def test_model_reductions():
    Nl, Nw, tI, tB = 3000, 400, 2e-7, 7e-8
    # hete with no CPUs is the GPU model, with no GPUs the CPU model
    assert pm.time_hete(Nl, Nw, 2, 40.0, 0, tI, tB) == pytest.approx(pm.time_gpu(Nl, Nw, 2, 40.0, tI, tB))
    assert pm.time_hete(Nl, Nw, 0, 40.0, 16, tI, tB) == pytest.approx(pm.time_cpu(Nl, Nw, 16, tI, tB))
    # alpha = 0 and no transfers: Eq. alpha is Eq. hete
    assert pm.time_alpha(Nl, Nw, 1, 40.0, 8, tI, tB, 0.0) == pytest.approx(pm.time_hete(Nl, Nw, 1, 40.0, 8, tI, tB))
    # t_B = beta t_I: Eq. beta is Eq. alpha
    beta = tB / tI
    assert pm.time_beta(Nl, Nw, 1, 40.0, 8, tI, 0.3, beta) == pytest.approx(
        pm.time_alpha(Nl, Nw, 1, 40.0, 8, tI, tB, 0.3))
    # one CPU worker, 2D (N_d = 1): Eq. cpu with C = 1 vs Eq. sequential's
    # interior term
    assert pm.time_cpu(Nl, Nw, 1, tI, 0.0) == pytest.approx(pm.time_seq(Nl, Nw, 1, tI, 0.0))
    # more workers never slow the interior term
    assert pm.time_hete(Nl, Nw, 1, 40.0, 8, tI, 0.0) < pm.time_hete(Nl, Nw, 1, 40.0, 0, tI, 0.0)


def test_boundary_cells():
    assert pm.boundary_cells([(10, 20, 1)]) == 60
    assert pm.boundary_cells([(4, 5, 6)]) == 2 * (20 + 24 + 30)
    assert pm.boundary_cells([(4, 5, 6), (4, 5, 6)]) == 4 * (20 + 24 + 30)


def _split_vs_whole(w, parts, steps):
    import numpy as np
    from paper_2305_18057_gb300 import workloads as wl
    from helpers import oracle_grid, oracle_states
    ws = wl.split_i(w, parts)
    assert sum(d[0] for d in ws.dims) == w.dims[0][0]
    g1, g2 = oracle_grid(w), oracle_grid(ws)
    U1, U2 = oracle_states(g1, w), oracle_states(g2, ws)
    R1 = g1.residual(U1)[0]
    R2 = np.concatenate(g2.residual(U2), axis=3)
    # an interface ghost holds exactly the neighbour's cells, so every face
    # sees the same operands: the decomposition changes no bit
    assert np.array_equal(R1, R2)
    for _ in range(steps):
        dt1, n1 = g1.rk_step(U1, cfl=w.cfl)
        dt2, n2 = g2.rk_step(U2, cfl=w.cfl)
        assert dt1 == dt2
        np.testing.assert_allclose(n2[0], n1[0], rtol=1e-12)
    whole = g1.interior(U1[0], 0)
    parts_ = np.concatenate([g2.interior(U, b) for b, U in enumerate(U2)], axis=3)
    assert np.array_equal(whole, parts_)


def test_split_ramp2d_is_exact():
    from paper_2305_18057_gb300 import workloads as wl
    _split_vs_whole(wl.ramp_2d(ni=96, nj=40, perturb=0.02), 5, 3)


def test_split_periodic3d_is_exact():
    from paper_2305_18057_gb300 import workloads as wl
    _split_vs_whole(wl.periodic_3d(n=21, nj=10, nk=8), 3, 2)


def test_fit_recovers_model():
    # exact model data (no noise): the fit returns its parameters
    samples = []
    for n in (1 << 20, 1 << 21, 1 << 22):
        for nb in (4096, 65536, 262144):
            samples.append((n, nb, n * 2e-9 + nb * 7e-10 + 3e-5))
    f = pm.fit(samples)
    assert f["t_I"] == pytest.approx(2e-9, rel=1e-9)
    assert f["t_B"] == pytest.approx(7e-10, rel=1e-7)
    assert f["beta"] == pytest.approx(0.35, rel=1e-7)
    assert f["max_rel_dev"] < 1e-9
