"""The sub-box form of the oracle used by the full-size GPU tests: the
residual of a sub-box whose ghosts come from the block's state (or from the
oracle's own rule on the block's physical boundary faces) is bitwise the
whole block's residual on those cells, and one step of an enlarged sub-box
is bitwise the whole block's step on the cells 6 or more cells inside its
cut faces (three stages of a two-cell stencil)."""
import numpy as np
import pytest

import oracle
from helpers import oracle_grid, oracle_states, oracle_subbox
from paper_2305_18057_gb300 import workloads as wl

CASES = {
    "periodic": lambda: wl.periodic_3d(n=24, nj=20, nk=18, seed=5),
    "ramp": lambda: wl.ramp_3d(ni=40, nj=24, nk=16, ratio=1.05, perturb=0.05),
}
BOXES = [((0, 0, 0), (9, 8, 7)), ((31, 16, 9), (40, 24, 16)), ((10, 5, 3), (21, 13, 11)), ((0, 16, 0), (12, 24, 16))]


@pytest.mark.parametrize("case", list(CASES))
def test_subbox_residual_is_the_block_residual(case):
    w = CASES[case]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    R = og.residual(Uo)[0]
    ni, nj, nk = w.dims[0]
    for lo, hi in BOXES:
        hi = (min(hi[0], ni), min(hi[1], nj), min(hi[2], nk))
        lo = tuple(min(a, b - 1) for a, b in zip(lo, hi))
        g, U = oracle_subbox(w, 0, lo, hi, w.U0[0])
        Rs = g.residual([U], fill=False)[0]
        assert np.array_equal(Rs, R[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]), (case, lo, hi)


def test_subbox_step_core_is_the_block_step():
    w = CASES["ramp"]()
    og = oracle_grid(w)
    Uo = oracle_states(og, w)
    dt = 0.5 * og.dt_min(Uo)
    og.rk_step(Uo, oracle.RK3_SSP, dt=dt)
    want = og.interior(Uo[0], 0)
    ni, nj, nk = w.dims[0]
    # a box on the inflow-wall corner: exact on its physical faces (inflow,
    # wall), 6 deep on its cut faces (the i and j ends, and both k faces,
    # periodic, whose ghosts are copied once)
    lo, hi = (0, 0, 0), (20, 16, nk)
    g, U = oracle_subbox(w, 0, lo, hi, w.U0[0])
    g.rk_step([U], oracle.RK3_SSP, dt=dt)
    got = g.interior(U, 0)
    core = (slice(None), slice(6, nk - 6), slice(0, hi[1] - 6), slice(0, hi[0] - 6))
    wcore = want[:, 6:nk - 6, 0:hi[1] - 6, 0:hi[0] - 6]
    assert wcore.size >= 5 * 4 * 10 * 14
    assert np.array_equal(got[core], wcore)
    # and the cut faces do matter: next to them the sub-box step differs
    assert not np.array_equal(got[:, :, :, -1], want[:, lo[2]:hi[2], lo[1]:hi[1], hi[0] - 1])
