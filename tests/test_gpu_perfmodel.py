"""The 1D decomposition of the performance model (Sec. 6) on the GPU: the
library gives the same bits whether a grid is one block or cut into P
i-blocks joined by interfaces (the oracle does too), and the decomposition
study returns a usable fit."""
import numpy as np
import pytest

from helpers import gpu_grid, gpu_states
from paper_2305_18057_gb300 import perfmodel as pm
from paper_2305_18057_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("make,parts", [
    (lambda: wl.ramp_2d(ni=150, nj=37, perturb=0.03), 5),
    (lambda: wl.periodic_3d(n=70, nj=19, nk=12), 3),
])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_split_is_exact_on_gpu(make, parts, precision):
    w = make()
    ws = wl.split_i(w, parts)
    g1, g2 = gpu_grid(w, precision=precision), gpu_grid(ws, precision=precision)
    U1, U2 = gpu_states(g1, w), gpu_states(g2, ws)
    R1 = [torch.empty((5, nk, nj, ni), dtype=torch.float64, device=U1[0].device) for ni, nj, nk in w.dims]
    R2 = [torch.empty((5, nk, nj, ni), dtype=torch.float64, device=U1[0].device) for ni, nj, nk in ws.dims]
    g1.residual(U1, R1)
    g2.residual(U2, R2)
    torch.cuda.synchronize()
    assert torch.equal(R1[0], torch.cat(R2, dim=3))
    for _ in range(3):
        g1.rk_step(U1, 1, cfl=w.cfl)
        g2.rk_step(U2, 1, cfl=w.cfl)
    torch.cuda.synchronize()
    whole = g1.download(U1[0], 0)
    cut = np.concatenate([g2.download(U, b) for b, U in enumerate(U2)], axis=3)
    assert np.array_equal(whole, cut)


def test_decomposition_study_small():
    def setup(w):
        g = gpu_grid(w)
        return g, gpu_states(g, w)
    ws = [wl.ramp_2d(ni=n, nj=128) for n in (256, 512)]
    rows, f = pm.decomposition_study(ws, (1, 4, 8), setup, steps=3, warmup=1)
    assert len(rows) == 6
    assert all(r["step_s"] > 0 for r in rows)
    assert f["t_I"] > 0 and np.isfinite(f["beta"])
