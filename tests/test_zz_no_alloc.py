"""sensei_residual_norms_noalloc: the residual norms for callers that cannot
allocate device memory (their device memory belongs to a host application's
pool, or they run inside a loop that must not risk an allocation).

It is checked against the workspace-based path it mirrors: sensei_residual
records the norms of the residual it writes, sensei_norms returns them; the
no-alloc call must give the same L2 and max norms of that same residual,
within the residual tolerance of the other tests (1e-11 relative), on two
calls in a row (the second call reuses the shared scratch the first left
behind).  This file is collected last so that a run stopping at the first
failure has run every other test first."""
import numpy as np
import pytest

from helpers import gpu_grid, gpu_states
from paper_2305_18057_gb300 import build as libbuild
from paper_2305_18057_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sensei():
    libbuild.build()
    from paper_2305_18057_gb300 import sensei as s
    s.load()
    return s


@pytest.mark.parametrize("dims", [(37, 19, 11), (64, 48, 40)])
def test_noalloc_norms_match_the_workspace_path(sensei, dims):
    ni, nj, nk = dims
    w = wl.periodic_3d(n=ni, nj=nj, nk=nk, seed=21)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    R = torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device)
    g.residual(Us, [R])
    _, l2_ref, linf_ref, _ = g.norms()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        l2, linf = sensei.sensei_residual_norms_noalloc(R.data_ptr(), ni, nj, nk, stream)
        np.testing.assert_allclose(l2, l2_ref, rtol=1e-11, err_msg=f"call {call}")
        np.testing.assert_allclose(linf, linf_ref, rtol=1e-11, err_msg=f"call {call}")


def test_noalloc_rejects_grids_beyond_its_scratch(sensei):
    R = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sensei.SenseiError) as e:
        sensei.sensei_residual_norms_noalloc(R.data_ptr(), 256, 256, 129, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == sensei.ERR_INVALID_ARG
    assert "8388608" in str(e.value)
