"""Thin ctypes binding of the C ABI in ``include/sensei.h`` (``libsensei.so``).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``csrc/``.  PyTorch supplies device memory and streams.  There is
no fallback: if the library cannot be loaded, every entry point raises.

Functions with the C names (``sensei_create_grid`` ...) take raw integers
(device addresses) and ctypes arrays, exactly like the C calls.  ``Grid`` is
a convenience owner of a grid, its workspace tensor and state tensors laid out
as ``sensei_state_layout`` says.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsensei.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_STATE = range(7)
FP64, FP32_FLUX, FP32_STORE, DF64 = 0, 1, 2, 3
BC_PERIODIC, BC_INFLOW, BC_EXTRAPOLATE, BC_SLIP_WALL, BC_INTERFACE, BC_EXTERNAL = range(6)
RK2_SSP, RK3_SSP, RK4_SSP2 = range(3)
LIM_NONE, LIM_MINMOD, LIM_VANLEER = range(3)
NV = 5

# every symbol include/sensei.h declares
EXPORTS = ("sensei_workspace_size", "sensei_create_grid", "sensei_destroy_grid", "sensei_state_layout",
           "sensei_set_bc", "sensei_fill_ghosts", "sensei_residual", "sensei_rk_step", "sensei_norms",
           "sensei_rk_step_local", "sensei_rk_steps", "sensei_step_graph_create", "sensei_steps_graph_create", "sensei_step_graph_launch", "sensei_step_graph_destroy", "sensei_autotune",
           "sensei_profile_enable", "sensei_profile_read", "sensei_profile_launches", "sensei_residual_norms_noalloc", "sensei_debug_set",
           "sensei_rk_stage", "sensei_face_exchange", "sensei_dt_min", "sensei_schedule",
           "sensei_host_create", "sensei_host_destroy", "sensei_host_set_bc", "sensei_host_layout",
           "sensei_host_state", "sensei_host_fill_ghosts", "sensei_host_residual", "sensei_host_dt_min",
           "sensei_host_stage", "sensei_host_face_exchange",
           "sensei_hetero_workspace_size", "sensei_hetero_create", "sensei_hetero_destroy", "sensei_hetero_upload",
           "sensei_hetero_download", "sensei_hetero_step",
           "sensei_last_error")


class BlockDesc(C.Structure):
    _fields_ = [("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int)]


class Scheme(C.Structure):
    _fields_ = [("gamma", C.c_double), ("limiter", C.c_int), ("kappa", C.c_double), ("eps", C.c_double),
                ("entropy_fix", C.c_double), ("precision", C.c_int), ("reconstruct_conserved", C.c_int),
                ("mu", C.c_double), ("prandtl", C.c_double)]


class Layout(C.Structure):
    _fields_ = [("stride_j", C.c_longlong), ("stride_k", C.c_longlong), ("stride_var", C.c_longlong),
                ("offset", C.c_longlong), ("elems", C.c_longlong), ("ghost_i", C.c_int), ("ghost_j", C.c_int),
                ("ghost_k", C.c_int), ("elem_bytes", C.c_int)]


class SenseiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sensei status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libsensei.so (built by ``paper_2305_18057_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2305_18057_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    L.sensei_workspace_size.argtypes = [C.POINTER(BlockDesc), C.c_int, C.POINTER(Scheme), C.POINTER(C.c_size_t)]
    L.sensei_create_grid.argtypes = [C.POINTER(BlockDesc), C.c_int, C.POINTER(vp), C.POINTER(Scheme), vp,
                                     C.c_size_t, vp, C.POINTER(vp)]
    L.sensei_destroy_grid.argtypes = [vp]
    L.sensei_state_layout.argtypes = [vp, C.c_int, C.POINTER(Layout)]
    L.sensei_set_bc.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp, C.c_int, C.c_int, C.c_int]
    L.sensei_fill_ghosts.argtypes = [vp, C.POINTER(vp), vp]
    L.sensei_residual.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), vp]
    L.sensei_rk_step.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_double, C.c_double, vp, vp]
    L.sensei_norms.argtypes = [vp, dp, dp, dp, vp]
    L.sensei_rk_step_local.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_double, vp, vp]
    L.sensei_step_graph_create.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_double, C.c_double, vp, vp,
                                           C.POINTER(vp)]
    L.sensei_rk_steps.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_int, C.c_double, C.c_double, vp, vp]
    L.sensei_steps_graph_create.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_int, C.c_double, C.c_double, vp, vp,
                                            C.POINTER(vp)]
    L.sensei_step_graph_launch.argtypes = [vp, vp]
    L.sensei_step_graph_destroy.argtypes = [vp]
    L.sensei_autotune.argtypes = [vp, C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(C.c_int), vp]
    L.sensei_profile_enable.argtypes = [vp, C.c_int]
    L.sensei_profile_read.argtypes = [vp, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.c_int]
    L.sensei_profile_launches.argtypes = [vp, dp, C.c_int, C.POINTER(C.c_int)]
    L.sensei_residual_norms_noalloc.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp, dp, vp]
    L.sensei_debug_set.argtypes = [vp, C.c_int, C.c_longlong]
    L.sensei_rk_stage.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_int, C.c_double, vp]
    ip = C.POINTER(C.c_int)
    L.sensei_schedule.argtypes = [vp, ip, ip, ip, ip]
    L.sensei_face_exchange.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_int, C.c_int, vp, C.c_int, vp]
    L.sensei_dt_min.argtypes = [vp, C.POINTER(vp), C.c_double, dp, vp]
    L.sensei_host_create.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.POINTER(Scheme), C.c_int, C.POINTER(vp)]
    L.sensei_host_destroy.argtypes = [vp]
    L.sensei_host_set_bc.argtypes = [vp, C.c_int, C.c_int, dp]
    L.sensei_host_layout.argtypes = [vp, C.POINTER(Layout)]
    L.sensei_host_state.argtypes = [vp]
    L.sensei_host_fill_ghosts.argtypes = [vp]
    L.sensei_host_residual.argtypes = [vp, dp]
    L.sensei_host_dt_min.argtypes = [vp, C.c_double, dp]
    L.sensei_host_stage.argtypes = [vp, C.c_int, C.c_int, C.c_double]
    L.sensei_host_face_exchange.argtypes = [vp, C.c_int, C.c_int, dp, C.c_int]
    L.sensei_hetero_workspace_size.argtypes = [C.POINTER(BlockDesc), C.POINTER(Scheme), C.c_int, C.POINTER(C.c_size_t)]
    L.sensei_hetero_create.argtypes = [C.POINTER(BlockDesc), dp, C.POINTER(Scheme), C.POINTER(C.c_int), dp, C.c_int,
                                       C.c_int, vp, C.c_size_t, vp, C.POINTER(vp)]
    L.sensei_hetero_destroy.argtypes = [vp]
    L.sensei_hetero_upload.argtypes = [vp, dp]
    L.sensei_hetero_download.argtypes = [vp, dp]
    L.sensei_hetero_step.argtypes = [vp, C.c_int, C.c_double, C.c_double, dp, dp]
    L.sensei_last_error.argtypes = []
    L.sensei_last_error.restype = C.c_char_p
    for name in EXPORTS[:-1]:
        getattr(L, name).restype = C.c_int
    L.sensei_host_state.restype = dp
    _lib = L
    return L


def _check(status):
    if status != OK:
        raise SenseiError(status, load().sensei_last_error().decode())
    return status


def _ptrs(addrs):
    arr = (C.c_void_p * len(addrs))()
    for n, a in enumerate(addrs):
        arr[n] = a
    return arr


# ------------------------------------------------------- the C entry points --

def sensei_workspace_size(blocks, scheme) -> int:
    b = (BlockDesc * len(blocks))(*[BlockDesc(*d) for d in blocks])
    n = C.c_size_t()
    _check(load().sensei_workspace_size(b, len(blocks), C.byref(scheme), C.byref(n)))
    return n.value


def sensei_create_grid(blocks, node_ptrs, scheme, workspace_ptr, workspace_bytes, stream_ptr):
    b = (BlockDesc * len(blocks))(*[BlockDesc(*d) for d in blocks])
    out = C.c_void_p()
    _check(load().sensei_create_grid(b, len(blocks), _ptrs(node_ptrs), C.byref(scheme), workspace_ptr,
                                     workspace_bytes, stream_ptr, C.byref(out)))
    return out.value


def sensei_destroy_grid(grid):
    return _check(load().sensei_destroy_grid(grid))


def sensei_state_layout(grid, block) -> Layout:
    lay = Layout()
    _check(load().sensei_state_layout(grid, block, C.byref(lay)))
    return lay


def sensei_set_bc(grid, block, face, bc_type, prim=None, nbr_block=-1, nbr_face=-1, orientation=0):
    p = (C.c_double * 5)(*prim) if prim is not None else None
    return _check(load().sensei_set_bc(grid, block, face, bc_type, p, nbr_block, nbr_face, orientation))


def sensei_fill_ghosts(grid, U_ptrs, stream_ptr):
    return _check(load().sensei_fill_ghosts(grid, _ptrs(U_ptrs), stream_ptr))


def sensei_residual(grid, U_ptrs, R_ptrs, src_ptrs, stream_ptr):
    s = _ptrs(src_ptrs) if src_ptrs is not None else None
    return _check(load().sensei_residual(grid, _ptrs(U_ptrs), _ptrs(R_ptrs), s, stream_ptr))


def sensei_rk_step(grid, U_ptrs, rk, cfl, dt, dt_used_ptr, stream_ptr):
    return _check(load().sensei_rk_step(grid, _ptrs(U_ptrs), rk, cfl, dt, dt_used_ptr, stream_ptr))


def sensei_norms(grid, stream_ptr, check=True):
    l2, linf, cons = (C.c_double * 5)(), (C.c_double * 5)(), (C.c_double * 5)()
    st = load().sensei_norms(grid, l2, linf, cons, stream_ptr)
    if check:
        _check(st)
    return st, np.array(l2[:]), np.array(linf[:]), np.array(cons[:])


def sensei_rk_step_local(grid, U_ptrs, rk, cfl, dt_min_ptr, stream_ptr):
    return _check(load().sensei_rk_step_local(grid, _ptrs(U_ptrs), rk, cfl, dt_min_ptr, stream_ptr))


def sensei_step_graph_create(grid, U_ptrs, rk, cfl, dt, dt_used_ptr, stream_ptr):
    out = C.c_void_p()
    _check(load().sensei_step_graph_create(grid, _ptrs(U_ptrs), rk, cfl, dt, dt_used_ptr, stream_ptr,
                                           C.byref(out)))
    return out.value


def sensei_rk_steps(grid, U_ptrs, nsteps, rk, cfl, dt, dt_used_ptr, stream_ptr):
    return _check(load().sensei_rk_steps(grid, _ptrs(U_ptrs), nsteps, rk, cfl, dt, dt_used_ptr, stream_ptr))


def sensei_steps_graph_create(grid, U_ptrs, nsteps, rk, cfl, dt, dt_used_ptr, stream_ptr):
    out = C.c_void_p()
    _check(load().sensei_steps_graph_create(grid, _ptrs(U_ptrs), nsteps, rk, cfl, dt, dt_used_ptr, stream_ptr,
                                            C.byref(out)))
    return out.value


def sensei_step_graph_launch(graph, stream_ptr):
    return _check(load().sensei_step_graph_launch(graph, stream_ptr))


def sensei_step_graph_destroy(graph):
    return _check(load().sensei_step_graph_destroy(graph))


def sensei_autotune(grid, U_ptrs, stream_ptr):
    """(kchunk, persistent) chosen by timing."""
    k, p = C.c_int(), C.c_int()
    _check(load().sensei_autotune(grid, _ptrs(U_ptrs), C.byref(k), C.byref(p), stream_ptr))
    return k.value, bool(p.value)


def sensei_profile_enable(grid, enable):
    return _check(load().sensei_profile_enable(grid, int(enable)))


def sensei_profile_read(grid, reset=True):
    """(stencil_ms, stencil_launches, kernel_launches) since the last reset."""
    ms, ns, nk = C.c_double(), C.c_longlong(), C.c_longlong()
    _check(load().sensei_profile_read(grid, C.byref(ms), C.byref(ns), C.byref(nk), int(reset)))
    return ms.value, ns.value, nk.value


def sensei_profile_launches(grid):
    """Durations (ms) of the stencil launches timed since the last reset, in order."""
    n = C.c_int()
    _check(load().sensei_profile_launches(grid, None, 0, C.byref(n)))
    buf = (C.c_double * max(n.value, 1))()
    _check(load().sensei_profile_launches(grid, buf, n.value, C.byref(n)))
    return list(buf[:n.value])


DEBUG_WAIT_LIMIT, DEBUG_TX_EXTRA, DEBUG_ITEM_ORDER = 1, 2, 3


def sensei_debug_set(grid, key, value):
    """Test hooks of the bounded device waits (see include/sensei.h)."""
    _check(load().sensei_debug_set(grid, int(key), int(value)))


def sensei_residual_norms_noalloc(R_ptr, ni, nj, nk, stream_ptr):
    """L2 and max norms of a dense residual R[5][nk][nj][ni] without any
    device allocation (for callers whose device memory is not theirs to
    allocate); returns (l2, linf)."""
    l2, linf = (C.c_double * 5)(), (C.c_double * 5)()
    _check(load().sensei_residual_norms_noalloc(R_ptr, ni, nj, nk, l2, linf, stream_ptr))
    return np.array(l2[:]), np.array(linf[:])


def sensei_last_error() -> str:
    return load().sensei_last_error().decode()


# ------------------------------------------------------------ convenience --

def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def sensei_schedule(grid) -> dict:
    v = [C.c_int() for _ in range(4)]
    _check(load().sensei_schedule(grid, *[C.byref(x) for x in v]))
    return {"kchunk": v[0].value, "persistent": bool(v[1].value), "order_by_cost": bool(v[2].value),
            "ctas_per_sm": v[3].value}


def sensei_rk_stage(grid, U_ptrs, rk, stage, dt, stream_ptr):
    return _check(load().sensei_rk_stage(grid, _ptrs(U_ptrs), rk, stage, dt, stream_ptr))


def sensei_face_exchange(grid, U_ptrs, block, stage, face, buf_ptr, unpack, stream_ptr):
    return _check(load().sensei_face_exchange(grid, _ptrs(U_ptrs), block, stage, face, buf_ptr, int(unpack),
                                              stream_ptr))


def sensei_dt_min(grid, U_ptrs, cfl, stream_ptr) -> float:
    out = C.c_double()
    _check(load().sensei_dt_min(grid, _ptrs(U_ptrs), cfl, C.byref(out), stream_ptr))
    return out.value


def sensei_host_create(ni, nj, nk, nodes, scheme, threads):
    out = C.c_void_p()
    X = np.ascontiguousarray(nodes, dtype=np.float64)
    _check(load().sensei_host_create(ni, nj, nk, _dptr(X), C.byref(scheme), threads, C.byref(out)))
    return out.value


def sensei_host_destroy(h):
    return _check(load().sensei_host_destroy(h))


def sensei_host_set_bc(h, face, bc_type, prim=None):
    p = _dptr(np.ascontiguousarray(prim, dtype=np.float64)) if prim is not None else None
    return _check(load().sensei_host_set_bc(h, face, bc_type, p))


def sensei_host_layout(h) -> Layout:
    lay = Layout()
    _check(load().sensei_host_layout(h, C.byref(lay)))
    return lay


def sensei_host_state(h):
    return load().sensei_host_state(h)


def sensei_host_fill_ghosts(h):
    return _check(load().sensei_host_fill_ghosts(h))


def sensei_host_residual(h, R: np.ndarray):
    return _check(load().sensei_host_residual(h, _dptr(R)))


def sensei_host_dt_min(h, cfl) -> float:
    out = C.c_double()
    _check(load().sensei_host_dt_min(h, cfl, C.byref(out)))
    return out.value


def sensei_host_stage(h, rk, stage, dt):
    return _check(load().sensei_host_stage(h, rk, stage, dt))


def sensei_host_face_exchange(h, stage, face, buf: np.ndarray, unpack):
    return _check(load().sensei_host_face_exchange(h, stage, face, _dptr(buf), int(unpack)))


def sensei_hetero_workspace_size(block, scheme, nk_host) -> int:
    n = C.c_size_t()
    _check(load().sensei_hetero_workspace_size(C.byref(BlockDesc(*block)), C.byref(scheme), nk_host, C.byref(n)))
    return n.value


def sensei_hetero_create(block, nodes, scheme, bc_types, bc_prims, nk_host, threads, ws_ptr, ws_bytes, stream_ptr):
    out = C.c_void_p()
    X = np.ascontiguousarray(nodes, dtype=np.float64)
    bt = (C.c_int * 6)(*bc_types)
    bp = _dptr(np.ascontiguousarray(bc_prims, dtype=np.float64)) if bc_prims is not None else None
    _check(load().sensei_hetero_create(C.byref(BlockDesc(*block)), _dptr(X), C.byref(scheme), bt, bp, nk_host,
                                       threads, ws_ptr, ws_bytes, stream_ptr, C.byref(out)))
    return out.value


def sensei_hetero_destroy(h):
    return _check(load().sensei_hetero_destroy(h))


def sensei_hetero_upload(h, U: np.ndarray):
    return _check(load().sensei_hetero_upload(h, _dptr(U)))


def sensei_hetero_download(h, U: np.ndarray):
    return _check(load().sensei_hetero_download(h, _dptr(U)))


def sensei_hetero_step(h, rk, cfl, dt=0.0):
    dt_used = C.c_double()
    times = (C.c_double * 4)()
    _check(load().sensei_hetero_step(h, rk, cfl, dt, C.byref(dt_used), times))
    return dt_used.value, list(times)


class HostBlock:
    """Owner of one host-worker block (the host share of co-execution): its
    state as a numpy view of the worker's own array."""

    def __init__(self, dims, nodes, gamma=1.4, limiter=LIM_VANLEER, kappa=1.0 / 3.0, eps=1.0, entropy_fix=0.1,
                 reconstruct_conserved=False, threads=1):
        self.dims = tuple(dims)
        ni, nj, nk = self.dims
        self.scheme = Scheme(gamma=gamma, limiter=limiter, kappa=kappa, eps=eps, entropy_fix=entropy_fix,
                             precision=FP64, reconstruct_conserved=int(reconstruct_conserved), mu=0.0, prandtl=0.72)
        self.handle = sensei_host_create(ni, nj, nk, nodes, self.scheme, threads)
        self.layout = sensei_host_layout(self.handle)
        ptr = sensei_host_state(self.handle)
        self.U = np.ctypeslib.as_array(ptr, shape=(self.layout.elems,))

    def interior(self):
        ni, nj, nk = self.dims
        L = self.layout
        return np.lib.stride_tricks.as_strided(self.U[L.offset:], shape=(5, nk, nj, ni),
                                               strides=(8 * L.stride_var, 8 * L.stride_k, 8 * L.stride_j, 8))

    def set_bc(self, face, bc_type, prim=None):
        sensei_host_set_bc(self.handle, face, bc_type, prim)

    def residual(self):
        ni, nj, nk = self.dims
        R = np.zeros((5, nk, nj, ni))
        sensei_host_residual(self.handle, R)
        return R

    def dt_min(self, cfl):
        return sensei_host_dt_min(self.handle, cfl)

    def step(self, rk, dt):
        for s in range(RK_STAGES[rk]):
            sensei_host_stage(self.handle, rk, s, dt)

    def close(self):
        if self.handle:
            sensei_host_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


RK_STAGES = {RK2_SSP: 2, RK3_SSP: 3, RK4_SSP2: 4}


class Hetero:
    """Owner of a co-execution driver (one block; the last nk_host k-planes
    on host threads, the rest on the GPU) and its device workspace."""

    def __init__(self, dims, nodes, bcs, nk_host, threads, gamma=1.4, limiter=LIM_VANLEER, kappa=1.0 / 3.0,
                 eps=1.0, entropy_fix=0.1, reconstruct_conserved=False):
        import torch
        self.torch = torch
        self.dims = tuple(dims)
        self.scheme = Scheme(gamma=gamma, limiter=limiter, kappa=kappa, eps=eps, entropy_fix=entropy_fix,
                             precision=FP64, reconstruct_conserved=int(reconstruct_conserved), mu=0.0, prandtl=0.72)
        nbytes = sensei_hetero_workspace_size(self.dims, self.scheme, nk_host)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        wsp = (base + 255) // 256 * 256
        types = [bc[0] for bc in bcs]
        prims = np.zeros((6, 5))
        for f, bc in enumerate(bcs):
            if bc[1] is not None:
                prims[f] = bc[1]
        self.stream = torch.cuda.current_stream()
        self.handle = sensei_hetero_create(self.dims, nodes, self.scheme, types, prims, nk_host, threads, wsp,
                                           nbytes, self.stream.cuda_stream)

    def upload(self, U):
        sensei_hetero_upload(self.handle, np.ascontiguousarray(U, dtype=np.float64))

    def download(self):
        ni, nj, nk = self.dims
        U = np.zeros((5, nk, nj, ni))
        sensei_hetero_download(self.handle, U)
        return U

    def step(self, rk=RK3_SSP, cfl=0.5, dt=0.0):
        return sensei_hetero_step(self.handle, rk, cfl, dt)

    def close(self):
        if self.handle:
            sensei_hetero_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StepGraph:
    def __init__(self, handle, grid):
        self.handle = handle
        self.grid = grid

    def launch(self, stream=None):
        sensei_step_graph_launch(self.handle, (stream or self.grid.stream).cuda_stream)

    def close(self):
        if self.handle:
            sensei_step_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """A grid on the current CUDA device with its workspace and state tensors.

    blocks: [(ni, nj, nk)], nodes: [(3, nk+1, nj+1, ni+1) float64 array or
    tensor].  ``scheme`` keys: gamma, limiter, kappa, eps, entropy_fix,
    precision, reconstruct_conserved.
    """

    def __init__(self, blocks, nodes, stream=None, **scheme):
        import torch
        self.torch = torch
        self.blocks = [tuple(int(v) for v in d) for d in blocks]
        self.scheme = Scheme(scheme.get("gamma", 1.4), scheme.get("limiter", LIM_VANLEER),
                             scheme.get("kappa", 1.0 / 3.0), scheme.get("eps", 1.0), scheme.get("entropy_fix", 0.1),
                             scheme.get("precision", FP64), int(scheme.get("reconstruct_conserved", 0)),
                             scheme.get("mu", 0.0), scheme.get("prandtl", 0.72))
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ws_bytes = sensei_workspace_size(self.blocks, self.scheme)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.dev)
        self._nodes = [torch.as_tensor(X, dtype=torch.float64).to(self.dev).contiguous() for X in nodes]
        self.handle = sensei_create_grid(self.blocks, [X.data_ptr() for X in self._nodes], self.scheme,
                                         self.workspace.data_ptr(), self.ws_bytes, self.stream.cuda_stream)
        self.layouts = [sensei_state_layout(self.handle, b) for b in range(len(self.blocks))]

    def close(self):
        if getattr(self, "handle", None):
            sensei_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def sptr(self):
        return self.stream.cuda_stream

    def set_bc(self, block, face, bc_type, prim=None, nbr=-1, nbr_face=-1):
        sensei_set_bc(self.handle, block, face, bc_type, prim, nbr, nbr_face, 0)

    def new_state(self, block):
        return self.torch.zeros(self.layouts[block].elems, dtype=self.torch.float64, device=self.dev)

    def interior_view(self, U, block):
        """(5, nk, nj, ni) view of a state tensor's interior cells."""
        ni, nj, nk = self.blocks[block]
        L = self.layouts[block]
        return U.as_strided((5, nk, nj, ni), (L.stride_var, L.stride_k, L.stride_j, 1), L.offset)

    def upload(self, U, block, interior):
        self.interior_view(U, block).copy_(self.torch.as_tensor(interior, dtype=self.torch.float64))

    def download(self, U, block):
        return self.interior_view(U, block).cpu().numpy().copy()

    def fill_ghosts(self, Us):
        sensei_fill_ghosts(self.handle, [U.data_ptr() for U in Us], self.sptr)

    def residual(self, Us, Rs, srcs=None):
        sensei_residual(self.handle, [U.data_ptr() for U in Us], [R.data_ptr() for R in Rs],
                        [s.data_ptr() for s in srcs] if srcs is not None else None, self.sptr)

    def rk_step(self, Us, rk=RK3_SSP, cfl=0.5, dt=0.0, dt_used=None):
        sensei_rk_step(self.handle, [U.data_ptr() for U in Us], rk, cfl, dt,
                       dt_used.data_ptr() if dt_used is not None else None, self.sptr)

    def rk_steps(self, Us, nsteps, rk=RK3_SSP, cfl=0.5, dt=0.0, dt_used=None):
        """nsteps rk_step calls in one (dt_used: a device tensor of nsteps doubles)."""
        sensei_rk_steps(self.handle, [U.data_ptr() for U in Us], nsteps, rk, cfl, dt,
                        dt_used.data_ptr() if dt_used is not None else None, self.sptr)

    def norms(self, check=True):
        return sensei_norms(self.handle, self.sptr, check=check)

    def rk_step_local(self, Us, rk=RK3_SSP, cfl=0.5, dt_min=None):
        sensei_rk_step_local(self.handle, [U.data_ptr() for U in Us], rk, cfl,
                             dt_min.data_ptr() if dt_min is not None else None, self.sptr)

    def step_graph(self, Us, rk=RK3_SSP, cfl=0.5, dt=0.0, dt_used=None):
        """A replayable CUDA graph of one rk_step on these states."""
        h = sensei_step_graph_create(self.handle, [U.data_ptr() for U in Us], rk, cfl, dt,
                                     dt_used.data_ptr() if dt_used is not None else None, self.sptr)
        return StepGraph(h, self)

    def steps_graph(self, Us, nsteps, rk=RK3_SSP, cfl=0.5, dt=0.0, dt_used=None):
        """A replayable CUDA graph of rk_steps(nsteps) on these states."""
        h = sensei_steps_graph_create(self.handle, [U.data_ptr() for U in Us], nsteps, rk, cfl, dt,
                                      dt_used.data_ptr() if dt_used is not None else None, self.sptr)
        return StepGraph(h, self)

    def autotune(self, Us):
        return sensei_autotune(self.handle, [U.data_ptr() for U in Us], self.sptr)

    def schedule(self):
        return sensei_schedule(self.handle)

    def debug_set(self, key, value):
        sensei_debug_set(self.handle, key, value)

    def profile(self, enable=True):
        sensei_profile_enable(self.handle, enable)

    def profile_read(self, reset=True):
        return sensei_profile_read(self.handle, reset)

    def profile_launches(self):
        return sensei_profile_launches(self.handle)
