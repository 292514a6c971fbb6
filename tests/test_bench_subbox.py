"""The bench's one-step oracle comparison on CPU: the sampled sub-boxes of
every workload shape lie inside their block (2D workloads keep their one
plane), and the oracle's step on a sub-box reproduces, on the box's core,
its step on the whole block (the cut faces' ghosts come from the state,
six margin cells keep the core away from them)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from helpers import oracle_grid, oracle_states  # noqa: E402
from paper_2305_18057_gb300 import workloads as wl  # noqa: E402
import oracle  # noqa: E402


@pytest.mark.parametrize("w", [wl.advection_2d(n=48), wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05),
                               wl.periodic_3d(n=24, nj=24, nk=24, seed=8)],
                         ids=["advection2d", "ramp2d", "periodic3d"])
def test_core_boxes_fit_their_blocks(w):
    boxes = bench._core_boxes(w)
    assert len(boxes) == 4
    for b, lo, hi in boxes:
        dims = w.dims[b]
        for d in range(3):
            assert 0 <= lo[d] < hi[d] <= dims[d]
        if dims[2] == 1:
            assert (lo[2], hi[2]) == (0, 1)
        else:
            assert hi[2] - lo[2] == 22


def test_subbox_step_matches_the_whole_block_2d():
    w = wl.ramp_2d(ni=70, nj=33, ratio=1.03, perturb=0.05)
    og = oracle_grid(w)
    U = oracle_states(og, w)[0]
    dt = 1e-6
    start = og.interior(U, 0).copy()
    og.rk_step([U], oracle.RK3_SSP, dt=dt)
    whole = og.interior(U, 0) - start   # the step's increment, whole block
    for b, lo, hi in bench._core_boxes(w):
        before, after = bench._oracle_subbox_step(w, b, lo, hi, dt)
        m = 6
        want = whole[:, :, lo[1] + m:hi[1] - m, lo[0] + m:hi[0] - m]
        got = after - before
        assert got.shape == want.shape
        scale = np.abs(want).max()
        assert scale > 1e-12 * np.abs(start).max()   # the step moves these cells
        assert np.abs(got - want).max() <= 1e-9 * scale
