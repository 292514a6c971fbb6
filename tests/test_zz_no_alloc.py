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

from helpers import gpu_grid, gpu_states, oracle_grid, oracle_states
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


def test_noalloc_norms_match_the_oracle(sensei):
    """The no-alloc norms of the GPU residual against the oracle's norms of
    its own residual of the same state (residual tolerance, 1e-11)."""
    ni, nj, nk = 37, 19, 11
    w = wl.periodic_3d(n=ni, nj=nj, nk=nk, seed=23)
    g = gpu_grid(w)
    Us = gpu_states(g, w)
    R = torch.empty((5, nk, nj, ni), dtype=torch.float64, device=Us[0].device)
    g.residual(Us, [R])
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    Ro = og.residual(Uo)
    l2_o, linf_o, _ = og.norms(Ro, Uo)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        l2, linf = sensei.sensei_residual_norms_noalloc(R.data_ptr(), ni, nj, nk, stream)
        np.testing.assert_allclose(l2, l2_o, rtol=1e-11, err_msg=f"call {call}")
        np.testing.assert_allclose(linf, linf_o, rtol=1e-11, err_msg=f"call {call}")


def test_noalloc_at_its_largest_size(sensei):
    """Exactly 8,388,608 cells (all 2048 partial slots, each finaliser lane
    striding over 64 of them) against an FP64 torch reduction of the same
    seeded dense array, on two calls in a row."""
    ni, nj, nk = 256, 256, 128
    gen = torch.Generator(device="cpu").manual_seed(2305)
    Rh = torch.randn((5, nk, nj, ni), dtype=torch.float64, generator=gen)
    Rh *= torch.tensor([1.0, 3.0, 1e-3, 1e4, 0.5], dtype=torch.float64).view(5, 1, 1, 1)
    R = Rh.cuda()
    l2_ref = torch.sqrt((Rh * Rh).reshape(5, -1).mean(dim=1)).numpy()
    linf_ref = Rh.abs().reshape(5, -1).amax(dim=1).numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        l2, linf = sensei.sensei_residual_norms_noalloc(R.data_ptr(), ni, nj, nk, stream)
        np.testing.assert_allclose(l2, l2_ref, rtol=1e-11, err_msg=f"call {call}")
        np.testing.assert_array_equal(linf, linf_ref, err_msg=f"call {call}")


def test_noalloc_reports_a_nan_residual(sensei):
    """A NaN entry of one variable makes both of its norms NaN; the other
    variables' norms are unaffected."""
    ni, nj, nk = 64, 48, 40
    gen = torch.Generator(device="cpu").manual_seed(7)
    Rh = torch.randn((5, nk, nj, ni), dtype=torch.float64, generator=gen)
    Rh[2, 17, 5, 33] = float("nan")
    R = Rh.cuda()
    l2, linf = sensei.sensei_residual_norms_noalloc(R.data_ptr(), ni, nj, nk, torch.cuda.current_stream().cuda_stream)
    assert np.isnan(l2[2]) and np.isnan(linf[2])
    keep = [0, 1, 3, 4]
    np.testing.assert_allclose(l2[keep], torch.sqrt((Rh[keep] ** 2).reshape(4, -1).mean(dim=1)).numpy(), rtol=1e-11)
    np.testing.assert_array_equal(linf[keep], Rh[keep].abs().reshape(4, -1).amax(dim=1).numpy())
