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


def oracle_subbox(w: wl.Workload, b, lo, hi, U_int):
    """The oracle on the cells lo <= (i, j, k) < hi of 3D block b, with the
    ghosted state taken from U_int (the block's interior state, (5, nk, nj,
    ni)): ghost cells that are cells of the block, or its wrapped cells across
    a periodic face, are copied; the ghosts of sub-box faces lying on a
    non-periodic boundary face of the block are filled by the oracle's own
    rule for that face; the other faces get no rule, so their ghosts stay as
    copied.  Returns (grid, ghosted state)."""
    ni, nj, nk = w.dims[b]
    assert nk > 1, "3D blocks only"
    (i0, j0, k0), (i1, j1, k1) = lo, hi
    faces = w.bcs[b]
    X = np.ascontiguousarray(w.nodes[b][:, k0:k1 + 1, j0:j1 + 1, i0:i1 + 1])
    g = oracle.OracleGrid([(i1 - i0, j1 - j0, k1 - k0)], [X], gamma=w.gamma, limiter=wl.LIMITERS[w.limiter],
                          kappa=w.kappa, eps=w.eps, fix=w.fix, mu=w.mu, prandtl=w.prandtl)

    def rng(a0, a1, n, periodic):
        r = np.arange(a0 - oracle.NG, a1 + oracle.NG)
        return r % n if periodic else np.clip(r, 0, n - 1)

    per = [faces[2 * d].type == wl.PERIODIC for d in range(3)]
    ii, jj, kk = rng(i0, i1, ni, per[0]), rng(j0, j1, nj, per[1]), rng(k0, k1, nk, per[2])
    U = np.ascontiguousarray(U_int[:, kk[:, None, None], jj[None, :, None], ii[None, None, :]])
    on_face = [i0 == 0, i1 == ni, j0 == 0, j1 == nj, k0 == 0, k1 == nk]
    for f in range(6):
        bc = faces[f]
        if on_face[f] and bc.type != wl.PERIODIC:
            assert bc.type != wl.INTERFACE, "single-block boundaries only"
            g.set_bc(0, f, bc.type, bc.prim)
    g.fill_ghosts([U])
    return g, U
