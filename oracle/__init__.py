"""Plain FP64 CPU oracle for the SENSEI explicit residual + Runge-Kutta path
(Euler, or Navier-Stokes with mu > 0).

TEST INFRASTRUCTURE.  The oracle restates arXiv 2305.18057 Sec. 2-3 and the
MUSCL paragraph of Sec. 5 in plain C (``sensei_oracle.c``, IEEE double,
``-ffp-contract=off``); this module compiles it with gcc and wraps it with
ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library
in ``paper_2305_18057_gb300`` and neither imports the other.

Array conventions (numpy, C order, float64):
  nodes  (3, nk+1, nj+1, ni+1)
  state  (5, nk+2gk, nj+4, ni+4), gk = 2 in 3D, 0 in 2D (nk == 1)
  residual / source (5, nk, nj, ni)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sensei_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libsensei_oracle.so")
# the same source compiled with a double that counts its operations
OPCOUNT_SRC = os.path.join(HERE, "opcount.cpp")
OPCOUNT_LIB = os.path.join(BUILD_DIR, "libsensei_oracle_opcount.so")

# boundary-condition, limiter and Runge-Kutta codes of the oracle
BC_PERIODIC, BC_INFLOW, BC_EXTRAPOLATE, BC_SLIP_WALL, BC_INTERFACE = 0, 1, 2, 3, 4
LIM_NONE, LIM_MINMOD, LIM_VANLEER = 0, 1, 2
RK2_SSP, RK3_SSP, RK4_SSP2 = 0, 1, 2
NV, NG = 5, 2

_lock = threading.Lock()
_libs = {}

_dp = C.POINTER(C.c_double)


def build(force: bool = False, counting: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libsensei_oracle.so`` (or,
    with ``counting``, its op-counting build ``libsensei_oracle_opcount.so``)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    out, srcs = (OPCOUNT_LIB, [OPCOUNT_SRC, SRC]) if counting else (LIB, [SRC])
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(f) for f in srcs)):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    if counting:
        cmd = ["g++", "-O2", "-std=c++17", "-fpermissive", "-w", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, OPCOUNT_SRC, "-lm"]
    else:
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, SRC, "-lm"]
    if counting:
        subprocess.run(cmd, check=True)
    elif subprocess.run(cmd, capture_output=True).returncode != 0:
        # a host compiler without OpenMP: the same source, one thread
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib(counting: bool = False):
    with _lock:
        if counting not in _libs:
            path = build(counting=counting)
            L = C.CDLL(path)
            L.ora_create.restype = C.c_void_p
            L.ora_create.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(_dp), C.c_double,
                                     C.c_int, C.c_double, C.c_double, C.c_int, C.c_double]
            L.ora_destroy.argtypes = [C.c_void_p]
            L.ora_set_bc.restype = C.c_int
            L.ora_set_bc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, _dp, C.c_int, C.c_int]
            L.ora_get_metrics.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp]
            L.ora_fill_ghosts.argtypes = [C.c_void_p, C.POINTER(_dp)]
            L.ora_residual.argtypes = [C.c_void_p, C.POINTER(_dp), C.POINTER(_dp), C.POINTER(_dp)]
            L.ora_dt_min.restype = C.c_double
            L.ora_dt_min.argtypes = [C.c_void_p, C.POINTER(_dp)]
            L.ora_norms.argtypes = [C.c_void_p, C.POINTER(_dp), C.POINTER(_dp), _dp]
            L.ora_rk_step.restype = C.c_double
            L.ora_rk_step.argtypes = [C.c_void_p, C.POINTER(_dp), C.POINTER(_dp), C.c_int,
                                      C.c_double, C.c_double, _dp]
            L.ora_rk_step_local.restype = C.c_double
            L.ora_rk_step_local.argtypes = [C.c_void_p, C.POINTER(_dp), C.POINTER(_dp), C.c_int, C.c_double, _dp]
            L.ora_rk_tableau.argtypes = [C.c_int, _dp, _dp, C.POINTER(C.c_int)]
            L.ora_set_viscosity.argtypes = [C.c_void_p, C.c_double, C.c_double]
            L.ora_euler_flux.argtypes = [C.c_double, _dp, _dp, _dp]
            L.ora_roe_flux.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp, _dp]
            L.ora_roe_jump.argtypes = [C.c_double, _dp, _dp, _dp, _dp]
            L.ora_muscl.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp]
            L.ora_psi.restype = C.c_double
            L.ora_psi.argtypes = [C.c_int, C.c_double]
            L.ora_cons_to_prim.argtypes = [C.c_double, _dp, _dp]
            L.ora_prim_to_cons.argtypes = [C.c_double, _dp, _dp]
            L.ora_set_threads.restype = C.c_int
            L.ora_set_threads.argtypes = [C.c_int]
            L.ora_set_threads(1)
            if counting:
                L.ora_opcount_reset.argtypes = []
                L.ora_opcount_get.argtypes = [C.POINTER(C.c_ulonglong)]
            _libs[counting] = L
    return _libs[counting]


def set_threads(n: int) -> int:
    """Host threads for the oracle's loops over k-planes (results are bitwise
    the same for every count); returns the count in effect (1 without
    OpenMP)."""
    return lib().ora_set_threads(int(n))


OPCOUNT_KINDS = ("add", "mul", "div", "sqrt", "cmp", "abs", "neg")


def opcount_reset():
    """Zero the operation counters of the op-counting build."""
    lib(counting=True).ora_opcount_reset()


def opcount_get():
    """Operations counted since the last reset: additions/subtractions,
    multiplications, divisions, square roots, comparisons, absolute values and
    min/max, negations."""
    out = (C.c_ulonglong * len(OPCOUNT_KINDS))()
    lib(counting=True).ora_opcount_get(out)
    return dict(zip(OPCOUNT_KINDS, (int(v) for v in out)))


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays are C-contiguous float64"
    return a.ctypes.data_as(_dp)


def _ptrs(arrs):
    arr = (_dp * len(arrs))()
    for n, a in enumerate(arrs):
        arr[n] = _ptr(a) if a is not None else _dp()
    return arr


def _vec(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ---------------------------------------------------------------- pointwise --

def euler_flux(W, S, gamma=1.4):
    """F_{i,n}(W) |S| for the area vector S (Eq. governing)."""
    W, S = _vec(W, 5), _vec(S, 3)
    F = np.zeros(5)
    lib().ora_euler_flux(gamma, _ptr(W), _ptr(S), _ptr(F))
    return F


def roe_flux(WL, WR, S, gamma=1.4, fix=0.1):
    WL, WR, S = _vec(WL, 5), _vec(WR, 5), _vec(S, 3)
    F = np.zeros(5)
    lib().ora_roe_flux(gamma, fix, _ptr(WL), _ptr(WR), _ptr(S), _ptr(F))
    return F


def roe_jump(WL, WR, S, gamma=1.4):
    WL, WR, S = _vec(WL, 5), _vec(WR, 5), _vec(S, 3)
    J = np.zeros(5)
    lib().ora_roe_jump(gamma, _ptr(WL), _ptr(WR), _ptr(S), _ptr(J))
    return J


def muscl(q4, limiter, kappa=1.0 / 3.0, eps=1.0):
    q4 = _vec(q4, 4)
    qL, qR = C.c_double(), C.c_double()
    lib().ora_muscl(limiter, kappa, eps, _ptr(q4), C.byref(qL), C.byref(qR))
    return qL.value, qR.value


def psi(limiter, r):
    return lib().ora_psi(limiter, float(r))


def cons_to_prim(Q, gamma=1.4):
    Q = _vec(Q, 5)
    W = np.zeros(5)
    lib().ora_cons_to_prim(gamma, _ptr(Q), _ptr(W))
    return W


def prim_to_cons(W, gamma=1.4):
    W = _vec(W, 5)
    Q = np.zeros(5)
    lib().ora_prim_to_cons(gamma, _ptr(W), _ptr(Q))
    return Q


def rk_tableau(rk):
    a = np.zeros(16)
    b = np.zeros(4)
    s = C.c_int()
    lib().ora_rk_tableau(rk, _ptr(a), _ptr(b), C.byref(s))
    return a.reshape(4, 4)[: s.value, : s.value].copy(), b[: s.value].copy()


# --------------------------------------------------------------------- grid --

class OracleGrid:
    """Multiblock structured grid held by the oracle (metrics computed in C)."""

    def __init__(self, dims, nodes, gamma=1.4, limiter=LIM_VANLEER, kappa=1.0 / 3.0, eps=1.0,
                 recon_conserved=False, fix=0.1, mu=0.0, prandtl=0.72, counting=False):
        self._L = lib(counting)
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.nodes = [np.ascontiguousarray(x, dtype=np.float64) for x in nodes]
        for (ni, nj, nk), X in zip(self.dims, self.nodes):
            assert X.shape == (3, nk + 1, nj + 1, ni + 1), (X.shape, (ni, nj, nk))
        flat = (C.c_int * (3 * len(self.dims)))(*[v for d in self.dims for v in d])
        self._h = self._L.ora_create(len(self.dims), flat, _ptrs(self.nodes), gamma, limiter, kappa,
                                   eps, int(recon_conserved), fix)
        self._L.ora_set_viscosity(self._h, mu, prandtl)
        self.gamma = gamma
        self.mu, self.prandtl = mu, prandtl

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.ora_destroy(h)
            self._h = None

    @property
    def nb(self):
        return len(self.dims)

    def gk(self, b):
        return 0 if self.dims[b][2] == 1 else NG

    def state_shape(self, b):
        ni, nj, nk = self.dims[b]
        return (NV, nk + 2 * self.gk(b), nj + 2 * NG, ni + 2 * NG)

    def alloc_state(self, b):
        return np.zeros(self.state_shape(b))

    def interior(self, U, b):
        ni, nj, nk = self.dims[b]
        g = self.gk(b)
        return U[:, g:g + nk, NG:NG + nj, NG:NG + ni]

    def set_bc(self, b, face, bc_type, prim=None, nbr=-1, nbr_face=-1):
        p = _vec(prim, 5) if prim is not None else None
        rc = self._L.ora_set_bc(self._h, b, face, bc_type, _ptr(p) if p is not None else _dp(), nbr, nbr_face)
        if rc != 0:
            raise ValueError(f"oracle rejected boundary condition (code {rc})")

    def metrics(self, b):
        ni, nj, nk = self.dims[b]
        Si = np.zeros((3, nk, nj, ni + 1))
        Sj = np.zeros((3, nk, nj + 1, ni))
        Sk = np.zeros((3, nk + 1, nj, ni))
        vol = np.zeros((nk, nj, ni))
        self._L.ora_get_metrics(self._h, b, _ptr(Si), _ptr(Sj), _ptr(Sk), _ptr(vol))
        return Si, Sj, Sk, vol

    def fill_ghosts(self, Us):
        self._L.ora_fill_ghosts(self._h, _ptrs(Us))

    def residual(self, Us, src=None, fill=True):
        """R_h of Eq. residual for every block; fills the ghost layers first."""
        if fill:
            self.fill_ghosts(Us)
        Rs = [np.zeros((NV,) + tuple(reversed(d))) for d in self.dims]
        srcp = _ptrs(src) if src is not None else None
        self._L.ora_residual(self._h, _ptrs(Us), _ptrs(Rs), srcp)
        return Rs

    def dt_min(self, Us, fill=True):
        if fill:
            self.fill_ghosts(Us)
        return self._L.ora_dt_min(self._h, _ptrs(Us))

    def norms(self, Rs, Us):
        out = np.zeros(15)
        self._L.ora_norms(self._h, _ptrs(Rs), _ptrs(Us), _ptr(out))
        return out[:5].copy(), out[5:10].copy(), out[10:].copy()

    def rk_step_local(self, Us, rk=RK3_SSP, cfl=0.5, src=None):
        """One step with local time stepping (every cell its own dt); returns
        (smallest dt, norms)."""
        out = np.zeros(15)
        srcp = _ptrs(src) if src is not None else None
        dt_min = self._L.ora_rk_step_local(self._h, _ptrs(Us), srcp, rk, cfl, _ptr(out))
        return dt_min, (out[:5].copy(), out[5:10].copy(), out[10:].copy())

    def rk_step(self, Us, rk=RK3_SSP, cfl=0.5, dt=0.0, src=None):
        """One Runge-Kutta step in place; returns (dt_used, (l2, linf, cons))."""
        out = np.zeros(15)
        srcp = _ptrs(src) if src is not None else None
        dt_used = self._L.ora_rk_step(self._h, _ptrs(Us), srcp, rk, cfl, dt, _ptr(out))
        return dt_used, (out[:5].copy(), out[5:10].copy(), out[10:].copy())
