"""The op-counting build of the oracle (oracle/opcount.cpp): the same source
with a counting double.  It must compute bit for bit what the plain build
computes, and the per-cell operation counts the bench reports beside its
roofline must be the ones it counts."""
import numpy as np
import pytest

import bench
import oracle
from helpers import oracle_states
from paper_2305_18057_gb300 import workloads as wl


def _grid(w, counting):
    g = oracle.OracleGrid(w.dims, w.nodes, gamma=w.gamma, limiter=wl.LIMITERS[w.limiter], kappa=w.kappa,
                          eps=w.eps, fix=w.fix, mu=w.mu, prandtl=w.prandtl, counting=counting)
    for b, faces in enumerate(w.bcs):
        for f in range(4 if w.dims[b][2] == 1 else 6):
            bc = faces[f]
            g.set_bc(b, f, bc.type, bc.prim, bc.nbr, bc.nbr_face)
    return g


@pytest.mark.parametrize("make", [lambda: wl.periodic_3d(n=12, nj=9, nk=7),
                                  lambda: wl.ramp_2d(ni=24, nj=12, ratio=1.05, perturb=0.05)])
def test_counting_build_is_bitwise_the_oracle(make):
    w = make()
    g0, g1 = _grid(w, False), _grid(w, True)
    U0, U1 = oracle_states(g0, w), oracle_states(g1, w)
    R0, R1 = g0.residual(U0), g1.residual(U1)
    assert all(np.array_equal(a, b) for a, b in zip(R0, R1))
    for _ in range(2):
        d0, _ = g0.rk_step(U0, oracle.RK3_SSP, cfl=0.5)
        d1, _ = g1.rk_step(U1, oracle.RK3_SSP, cfl=0.5)
        assert d0 == d1
    assert all(np.array_equal(a, b) for a, b in zip(U0, U1))


def test_counts_are_exact_and_match_the_bench():
    oracle.opcount_reset()
    assert oracle.opcount_get() == dict.fromkeys(oracle.OPCOUNT_KINDS, 0)
    w = wl.periodic_3d(n=24)
    g = _grid(w, True)
    U = oracle_states(g, w)
    oracle.opcount_reset()
    g.rk_step(U, oracle.RK3_SSP, cfl=0.5)
    c = oracle.opcount_get()
    n = 3 * int(np.prod(w.dims[0]))
    per = {k: round(v / n, 3) for k, v in c.items() if k != "neg"}
    assert per == bench.ORACLE_OPS_PER_CELL_STAGE
    assert c["neg"] == 0
    # the plain oracle does about twice the kernel's counted arithmetic
    arith = per["add"] + per["mul"] + per["div"] + per["sqrt"]
    kernel = bench.alg_flops_per_cell("vanleer", False, True, False)
    assert 1.5 * kernel < arith < 3.0 * kernel
