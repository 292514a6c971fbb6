"""Test helpers: build oracle grids from workloads, embed states."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2305_18057_gb300 import workloads as wl


def oracle_grid(w: wl.Workload, limiter=None, kappa=None, recon_conserved=False, fix=None):
    lim = wl.LIMITERS[limiter if limiter is not None else w.limiter]
    g = oracle.OracleGrid(w.dims, w.nodes, gamma=w.gamma, limiter=lim,
                          kappa=w.kappa if kappa is None else kappa, eps=w.eps,
                          recon_conserved=recon_conserved, fix=w.fix if fix is None else fix,
                          mu=w.mu, prandtl=w.prandtl)
    for b, faces in enumerate(w.bcs):
        nfaces = 4 if w.dims[b][2] == 1 else 6
        for f in range(nfaces):
            bc = faces[f]
            g.set_bc(b, f, bc.type, bc.prim, bc.nbr, bc.nbr_face)
    return g


def oracle_states(g: oracle.OracleGrid, w: wl.Workload, U0=None):
    Us = []
    for b in range(g.nb):
        U = g.alloc_state(b)
        g.interior(U, b)[...] = (w.U0 if U0 is None else U0)[b]
        Us.append(U)
    return Us


def rel_err(a, b, scale=None):
    a = np.asarray(a)
    b = np.asarray(b)
    s = np.max(np.abs(b)) if scale is None else scale
    return float(np.max(np.abs(a - b)) / s) if s > 0 else float(np.max(np.abs(a - b)))


def gpu_grid(w: wl.Workload, limiter=None, precision=0, kappa=None, recon_conserved=False, fix=None):
    """The CUDA library's grid for a workload (same scheme as oracle_grid)."""
    from paper_2305_18057_gb300 import sensei
    lim = wl.LIMITERS[limiter if limiter is not None else w.limiter]
    g = sensei.Grid(w.dims, w.nodes, gamma=w.gamma, limiter=lim, kappa=w.kappa if kappa is None else kappa,
                    eps=w.eps, entropy_fix=w.fix if fix is None else fix, precision=precision,
                    reconstruct_conserved=recon_conserved, mu=w.mu, prandtl=w.prandtl)
    for b, faces in enumerate(w.bcs):
        nfaces = 4 if w.dims[b][2] == 1 else 6
        for f in range(nfaces):
            bc = faces[f]
            g.set_bc(b, f, bc.type, bc.prim, bc.nbr, bc.nbr_face)
    return g


def gpu_states(g, w: wl.Workload, U0=None):
    Us = []
    for b in range(len(w.dims)):
        U = g.new_state(b)
        g.upload(U, b, (w.U0 if U0 is None else U0)[b])
        Us.append(U)
    return Us


def per_var_rel(got, want, floor_frac=1e-3):
    """max over variables of max|got - want| / scale_v, with scale_v = max|want_v|
    floored at floor_frac * max over all variables (for identically-zero variables)."""
    got = np.asarray(got)
    want = np.asarray(want)
    gmax = np.abs(want).max()
    worst = 0.0
    for v in range(want.shape[0]):
        scale = max(np.abs(want[v]).max(), floor_frac * gmax, 1e-300)
        worst = max(worst, float(np.abs(got[v] - want[v]).max() / scale))
    return worst
