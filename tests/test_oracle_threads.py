"""The oracle's host threads change no result: with OpenMP over the loops of
independent k-planes (every face flux, the per-cell sums of Eq. residual,
the Runge-Kutta updates, the local time steps) and serial reductions, a run
on several threads is bitwise the single-thread run."""
import numpy as np
import pytest

import oracle
from helpers import oracle_grid, oracle_states
from paper_2305_18057_gb300 import workloads as wl


def _run(w, threads, local=False):
    oracle.set_threads(threads)
    try:
        g = oracle_grid(w)
        Us = oracle_states(g, w)
        R0 = g.residual(Us)
        outs = []
        for _ in range(2):
            if local:
                outs.append(g.rk_step_local(Us, oracle.RK3_SSP, cfl=0.5))
            else:
                outs.append(g.rk_step(Us, oracle.RK3_SSP, cfl=0.5))
        return R0, [U.copy() for U in Us], outs
    finally:
        oracle.set_threads(1)


@pytest.mark.parametrize("case", ["periodic", "lattice", "ramp2d_local"])
def test_threads_bitwise(case):
    if oracle.set_threads(4) < 2:
        oracle.set_threads(1)
        pytest.skip("oracle built without OpenMP")
    oracle.set_threads(1)
    if case == "periodic":
        w, local = wl.periodic_3d(n=20, nj=13, nk=17, seed=5), False
    elif case == "lattice":
        w, local = wl.lattice_3d(sizes=(6, 8, 10), nblk=(2, 2, 2), seed=3, perturb=0.05), False
    else:
        w, local = wl.ramp_2d(ni=40, nj=24, perturb=0.05, seed=6), True
    R1, U1, o1 = _run(w, 1, local)
    R4, U4, o4 = _run(w, 4, local)
    for a, b in zip(R1, R4):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(U1, U4):
        np.testing.assert_array_equal(a, b)
    for (dt1, n1), (dt4, n4) in zip(o1, o4):
        assert dt1 == dt4
        for x, y in zip(n1, n4):
            np.testing.assert_array_equal(x, y)
