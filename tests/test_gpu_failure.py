"""Failure detection without a GPU fault: the FP32 stencil's bounded waits on
its bulk tile copies are made to run out through the test hook (every tile
phase expects more bytes than arrive), the device error word reports
SENSEI_ERR_TIMEOUT through sensei_norms, and the context stays usable: the
next residual, hooks cleared, is bitwise the one before."""
import pytest

from helpers import gpu_grid, gpu_states
from paper_2305_18057_gb300 import sensei, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precision", ["fp32_flux", "fp32_store"])
def test_bounded_wait_timeout_is_reported_and_the_context_survives(precision):
    w = wl.periodic_3d(n=40, nj=19, nk=9, seed=3)
    g = gpu_grid(w, precision={"fp32_flux": sensei.FP32_FLUX, "fp32_store": sensei.FP32_STORE}[precision])
    Us = gpu_states(g, w)
    Rs = [torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device) for ni, nj, nk in w.dims]
    g.residual(Us, Rs)
    torch.cuda.synchronize()
    ref = Rs[0].clone()
    g.norms()
    # waits of about 2 ms (2^22 cycles) that cannot complete
    g.debug_set(sensei.DEBUG_WAIT_LIMIT, 1 << 22)
    g.debug_set(sensei.DEBUG_TX_EXTRA, 16)
    Rs[0].fill_(0.0)
    g.residual(Us, Rs)
    with pytest.raises(sensei.SenseiError) as e:
        g.norms()
    assert e.value.status == sensei.ERR_TIMEOUT
    g.debug_set(sensei.DEBUG_TX_EXTRA, 0)
    g.debug_set(sensei.DEBUG_WAIT_LIMIT, 0)
    g.residual(Us, Rs)
    torch.cuda.synchronize()
    assert torch.equal(Rs[0], ref)
    g.norms()
