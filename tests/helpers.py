"""Test helpers: build oracle grids from workloads, embed states."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2305_18057_gb300 import workloads as wl


def oracle_grid(w: wl.Workload, limiter=None, kappa=None, recon_conserved=False, fix=None):
    lim = wl.LIMITERS[limiter if limiter is not None else w.limiter]
    g = oracle.OracleGrid(w.dims, w.nodes, gamma=w.gamma, limiter=lim,
                          kappa=w.kappa if kappa is None else kappa, eps=w.eps,
                          recon_conserved=recon_conserved, fix=w.fix if fix is None else fix)
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
