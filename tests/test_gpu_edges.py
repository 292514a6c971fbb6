"""Edge cases of the GPU path against the oracle: blocks at the minimum
extent (two cells, the ghost depth) joined by interfaces in every direction,
and single blocks one cell short of, exactly at and one cell past the tile
sizes (32 x 8), in the three precisions."""
import numpy as np
import pytest

import oracle
from helpers import gpu_grid, gpu_states, oracle_grid, oracle_states, per_var_rel
from paper_2305_18057_gb300 import sensei, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PREC = {"fp64": (sensei.FP64, 1e-11), "fp32_flux": (sensei.FP32_FLUX, 2e-4), "fp32_store": (sensei.FP32_STORE, 2e-4)}

CASES = {
    "thin_lattice": lambda: wl.lattice_3d(sizes=(2, 3), nblk=(2, 2, 2), seed=0, perturb=0.05),
    "tile_minus": lambda: wl.periodic_3d(n=31, nj=7, nk=5, seed=8),
    "tile_exact": lambda: wl.periodic_3d(n=32, nj=8, nk=4, seed=9),
    "tile_plus": lambda: wl.ramp_3d(ni=33, nj=9, nk=3, ratio=1.05, perturb=0.05),
    "thin_2d": lambda: wl.ramp_2d(ni=2, nj=2, perturb=0.05),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", list(PREC))
def test_edge_case_residual(case, prec):
    w = CASES[case]()
    precision, tol = PREC[prec]
    og = oracle_grid(w)
    Ro = og.residual(oracle_states(og, w))
    g = gpu_grid(w, precision=precision)
    Us = gpu_states(g, w)
    Rs = [torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device) for ni, nj, nk in w.dims]
    g.residual(Us, Rs)
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(Rs[b].cpu().numpy(), Ro[b]) < tol, (case, prec, b)


@pytest.mark.parametrize("case", ["thin_lattice", "tile_plus", "thin_2d"])
def test_edge_case_steps_fp64(case):
    w = CASES[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    dt_used = torch.zeros(1, dtype=torch.float64, device=Us[0].device)
    for _ in range(10):
        g.rk_step(Us, 1, cfl=0.5, dt_used=dt_used)
        og.rk_step(Uo, oracle.RK3_SSP, dt=dt_used.item())
    torch.cuda.synchronize()
    for b in range(len(w.dims)):
        assert per_var_rel(g.download(Us[b], b), og.interior(Uo[b], b)) < 1e-9, (case, b)
