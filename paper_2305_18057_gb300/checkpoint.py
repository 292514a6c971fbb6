"""Checkpoint and resume of a run: the interior FP64 states of every block
with the step count, the physical time and the grid description, in one
numpy .npz file written on the host.  Ghost cells are not stored: every
library call refills them, so a resumed run continues bitwise as if it had
not stopped (the library is deterministic: fixed-order reductions, exact
dt minimum)."""
from __future__ import annotations

import os

import numpy as np

FORMAT = 1


def save(path, dims, interiors, step=0, time=0.0, **meta):
    """Write the interior states (one (5, nk, nj, ni) float64 array per
    block) and the run's counters; the file appears atomically."""
    dims = np.asarray(dims, dtype=np.int64).reshape(-1, 3)
    assert len(interiors) == len(dims)
    arrays = {f"U{b}": np.ascontiguousarray(U, dtype=np.float64) for b, U in enumerate(interiors)}
    for b, (ni, nj, nk) in enumerate(dims):
        assert arrays[f"U{b}"].shape == (5, nk, nj, ni), (b, arrays[f"U{b}"].shape)
    extra = {f"meta_{k}": np.asarray(v) for k, v in meta.items()}
    tmp = f"{path}.{os.getpid()}.tmp.npz"
    np.savez(tmp, format=np.int64(FORMAT), dims=dims, step=np.int64(step), time=np.float64(time), **arrays, **extra)
    os.replace(tmp, path)


def load(path):
    """(dims, interiors, step, time, meta) from a checkpoint file."""
    with np.load(path) as f:
        if int(f["format"]) != FORMAT:
            raise ValueError(f"{path}: checkpoint format {int(f['format'])}, expected {FORMAT}")
        dims = [tuple(int(v) for v in d) for d in f["dims"]]
        interiors = [f[f"U{b}"].copy() for b in range(len(dims))]
        meta = {k[5:]: f[k] for k in f.files if k.startswith("meta_")}
        return dims, interiors, int(f["step"]), float(f["time"]), meta


def save_grid(path, grid, Us, step=0, time=0.0, **meta):
    """Checkpoint the states Us of a library grid (sensei.Grid)."""
    save(path, grid.blocks, [grid.download(U, b) for b, U in enumerate(Us)], step, time, **meta)


def load_grid(path, grid, Us):
    """Restore a checkpoint into the states Us of a grid with the same
    blocks; returns (step, time, meta)."""
    dims, interiors, step, time, meta = load(path)
    if [tuple(d) for d in dims] != [tuple(d) for d in grid.blocks]:
        raise ValueError(f"{path}: blocks {dims} do not match the grid's {grid.blocks}")
    for b, (U, X) in enumerate(zip(Us, interiors)):
        grid.upload(U, b, X)
    return step, time, meta
