"""Checkpoint/resume: the file round-trips bitwise (host), and a run stopped,
saved, reloaded into a fresh grid and continued equals the uninterrupted
run bitwise (GPU)."""
import numpy as np
import pytest

from paper_2305_18057_gb300 import checkpoint, workloads as wl


def test_checkpoint_roundtrip_is_bitwise(tmp_path):
    w = wl.lattice_3d(sizes=(3, 4, 5), nblk=(2, 2, 1), seed=2, perturb=0.05)
    path = str(tmp_path / "run.npz")
    checkpoint.save(path, w.dims, w.U0, step=17, time=0.125, cfl=0.5)
    dims, U, step, time, meta = checkpoint.load(path)
    assert dims == [tuple(d) for d in w.dims] and step == 17 and time == 0.125 and float(meta["cfl"]) == 0.5
    for a, b in zip(U, w.U0):
        assert a.dtype == np.float64 and np.array_equal(a, b)
    with pytest.raises(AssertionError):
        checkpoint.save(path, w.dims, w.U0[::-1])


@pytest.mark.gpu
def test_resume_continues_bitwise(tmp_path):
    torch = pytest.importorskip("torch")
    from helpers import gpu_grid, gpu_states
    w = wl.ramp_2d(ni=70, nj=33, perturb=0.05)
    g = gpu_grid(w)
    U = gpu_states(g, w)
    for _ in range(6):
        g.rk_step(U, 1, cfl=0.5)
    torch.cuda.synchronize()
    straight = [g.download(u, b) for b, u in enumerate(U)]
    g1 = gpu_grid(w)
    U1 = gpu_states(g1, w)
    for _ in range(3):
        g1.rk_step(U1, 1, cfl=0.5)
    path = str(tmp_path / "half.npz")
    checkpoint.save_grid(path, g1, U1, step=3)
    del g1, U1
    g2 = gpu_grid(w)
    U2 = gpu_states(g2, w)
    step, _, _ = checkpoint.load_grid(path, g2, U2)
    assert step == 3
    for _ in range(3):
        g2.rk_step(U2, 1, cfl=0.5)
    torch.cuda.synchronize()
    for b, u in enumerate(U2):
        assert np.array_equal(g2.download(u, b), straight[b])
