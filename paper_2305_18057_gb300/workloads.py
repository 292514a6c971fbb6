"""Seeded synthetic inputs: grids, initial states and boundary descriptions.

This module only *makes inputs*.  It holds none of the solver's arithmetic
(no flux, reconstruction, residual, time step or update); the one piece of
physics it uses is the ideal-gas relation that turns the seeded primitive
fields (rho, u, v, w, p) into the conserved vector Q of Eq. governing, so
that both the CUDA library and the CPU oracle start from the same bytes.
Both sides import it; it imports neither.

The paper's own workload, the supersonic flow through a simplified 2D 30-deg
inlet (Sec. 7), survives only as its inflow table (Mach 4, 12270 Pa, 217 K);
its geometry is in figures that are not available.  The grids here stand in
for it: a periodic Mach-2 advection box (2D), a Mach-4 compression ramp
(2D and 3D) with the paper's inflow state, a smooth curvilinear periodic cube
(3D), and a 4x4x4 lattice of uneven blocks around a ramp (3D multiblock).

Array conventions: nodes (3, nk+1, nj+1, ni+1); interior states
(5, nk, nj, ni); all float64, C order.  A 2D grid is one cell deep (nk == 1)
with its two node planes at z = 0 and z = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = 1.4
R_AIR = 287.0   # J/(kg K); the paper gives p, T and M but not the gas constant

# face numbering shared by both sides: imin, imax, jmin, jmax, kmin, kmax
IMIN, IMAX, JMIN, JMAX, KMIN, KMAX = range(6)
PERIODIC, INFLOW, EXTRAPOLATE, SLIP_WALL, INTERFACE = 0, 1, 2, 3, 4
LIMITERS = {"none": 0, "minmod": 1, "vanleer": 2}
RK_SCHEMES = {"rk2": 0, "rk3": 1, "rk4": 2}


@dataclasses.dataclass
class BC:
    type: int
    prim: tuple | None = None      # (rho, u, v, w, p) for INFLOW
    nbr: int = -1                  # neighbour block for INTERFACE
    nbr_face: int = -1


@dataclasses.dataclass
class Workload:
    name: str
    dims: list                      # [(ni, nj, nk)] per block
    nodes: list                     # [(3, nk+1, nj+1, ni+1)] per block
    U0: list                        # [(5, nk, nj, ni)] conserved, per block
    bcs: list                       # [[BC x 6]] per block
    limiter: str = "vanleer"
    rk: str = "rk3"
    cfl: float = 0.5
    steps: int = 100
    gamma: float = GAMMA
    kappa: float = 1.0 / 3.0
    eps: float = 1.0
    fix: float = 0.1
    mu: float = 0.0                 # dynamic viscosity of F_nu (0: Euler)
    prandtl: float = 0.72
    note: str = ""

    @property
    def cells(self) -> int:
        return int(sum(ni * nj * nk for ni, nj, nk in self.dims))


# --------------------------------------------------------------- states ----

def inlet_inflow(direction=(1.0, 0.0, 0.0), mach=4.0, p=12270.0, T=217.0):
    """Primitive (rho, u, v, w, p) of the paper's inflow table (Sec. 7,
    Table inlet_inflow: Mach 4, 12270 Pa, 217 K), with R = 287 J/(kg K)."""
    rho = p / (R_AIR * T)
    c = math.sqrt(GAMMA * R_AIR * T)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    u = mach * c * d
    return (rho, float(u[0]), float(u[1]), float(u[2]), p)


def normalized_freestream(mach, direction):
    """rho = 1, p = 1/gamma (sound speed 1), speed = mach along direction."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return (1.0, float(mach * d[0]), float(mach * d[1]), float(mach * d[2]), 1.0 / GAMMA)


def conserved(rho, u, v, w, p, gamma=GAMMA):
    """Conserved Q = (rho, rho u, rho v, rho w, rho e_t) from primitive fields."""
    rho, u, v, w, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, v, w, p))
    shape = np.broadcast_shapes(rho.shape, u.shape, v.shape, w.shape, p.shape)
    Q = np.empty((5,) + shape)
    Q[0] = rho
    Q[1] = rho * u
    Q[2] = rho * v
    Q[3] = rho * w
    Q[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return Q


def uniform_state(dims, prim, gamma=GAMMA, perturb=0.0, seed=0):
    """Conserved state of a uniform primitive state; with perturb > 0, rho and
    p are multiplied by 1 + perturb * U(-1, 1) and every velocity component
    gets perturb * |u| * U(-1, 1) (seeded), cell by cell."""
    ni, nj, nk = dims
    ones = np.ones((nk, nj, ni))
    rho, u, v, w, p = (c * ones for c in prim)
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        speed = math.sqrt(prim[1] ** 2 + prim[2] ** 2 + prim[3] ** 2)
        rho = rho * (1.0 + perturb * rng.uniform(-1, 1, ones.shape))
        p = p * (1.0 + perturb * rng.uniform(-1, 1, ones.shape))
        u = u + perturb * speed * rng.uniform(-1, 1, ones.shape)
        v = v + perturb * speed * rng.uniform(-1, 1, ones.shape)
        if nk > 1:
            w = w + perturb * speed * rng.uniform(-1, 1, ones.shape)
    return conserved(rho, u, v, w, p, gamma)


def cell_centres(X):
    """Mean of the 8 corner nodes of every cell: (3, nk, nj, ni)."""
    return 0.125 * (X[:, :-1, :-1, :-1] + X[:, :-1, :-1, 1:] + X[:, :-1, 1:, :-1] + X[:, :-1, 1:, 1:]
                    + X[:, 1:, :-1, :-1] + X[:, 1:, :-1, 1:] + X[:, 1:, 1:, :-1] + X[:, 1:, 1:, 1:])


# ---------------------------------------------------------------- grids ----

def cartesian_nodes(ni, nj, nk, lengths=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0)):
    """Uniform Cartesian nodes; a 2D grid (nk == 1) spans z in [0, 1]."""
    xs = origin[0] + lengths[0] * np.arange(ni + 1) / ni
    ys = origin[1] + lengths[1] * np.arange(nj + 1) / nj
    zs = origin[2] + (lengths[2] if nk > 1 else 1.0) * np.arange(nk + 1) / nk
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.ascontiguousarray(np.stack([Xg, Y, Z]))


def periodic_sine_nodes(ni, nj, nk, amplitude_cells=0.05, seed=0):
    """Smooth periodic curvilinear map of the unit cube (unit square x [0,1]
    in 2D): x_c = xi_c + A sin(2 pi (xi_a + phi)) sin(2 pi (xi_b + phi')),
    (a, b) the two other axes, phases seeded, A = amplitude_cells * spacing.
    The displacement is periodic, so the map tiles space."""
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0.0, 1.0, size=(3, 2))
    xi = np.arange(ni + 1) / ni
    eta = np.arange(nj + 1) / nj
    zeta = np.arange(nk + 1) / nk
    Zt, Et, Xi = np.meshgrid(zeta, eta, xi, indexing="ij")
    h = 1.0 / max(ni, nj, nk if nk > 1 else 1)
    A = amplitude_cells * h
    s = lambda t, ph: np.sin(2.0 * np.pi * (t + ph))
    if nk == 1:
        x = Xi + A * s(Et, phase[0, 0]) * s(Et, phase[0, 1] + 0.25)
        y = Et + A * s(Xi, phase[1, 0]) * s(Xi, phase[1, 1] + 0.25)
        z = Zt
    else:
        x = Xi + A * s(Et, phase[0, 0]) * s(Zt, phase[0, 1])
        y = Et + A * s(Zt, phase[1, 0]) * s(Xi, phase[1, 1])
        z = Zt + A * s(Xi, phase[2, 0]) * s(Et, phase[2, 1])
    return np.ascontiguousarray(np.stack([x, y, z]))


def geometric_spacing(n, ratio):
    """Node coordinates s_0..s_n on [0, 1], spacing growing by `ratio` away from s = 0."""
    if abs(ratio - 1.0) < 1e-15:
        return np.arange(n + 1) / n
    j = np.arange(n + 1, dtype=np.float64)
    return np.expm1(j * math.log(ratio)) / math.expm1(n * math.log(ratio))


def ramp_nodes(ni, nj, nk, length=2.0, height=1.0, corner=0.5, angle_deg=10.0, ratio=1.02, depth=1.0, stride=1):
    """Compression ramp: wall y_w(x) = max(0, x - corner) tan(angle), top wall
    at y = height, j-nodes geometric with `ratio` away from the ramp; k is an
    extrusion over `depth` (a single unit-depth cell layer in 2D).  With
    stride > 1 the grid is every stride-th node of the (stride*ni) x
    (stride*nj) x (stride*nk) grid (a node restriction)."""
    x = length * np.arange(stride * ni + 1)[::stride] / (stride * ni)
    yw = np.maximum(0.0, x - corner) * math.tan(math.radians(angle_deg))
    s = geometric_spacing(stride * nj, ratio)[::stride]
    zs = (depth if nk > 1 else 1.0) * np.arange(stride * nk + 1)[::stride] / (stride * nk)
    X = np.empty((3, nk + 1, nj + 1, ni + 1))
    X[0] = x[None, None, :]
    X[1] = yw[None, None, :] + (height - yw[None, None, :]) * s[None, :, None]
    X[2] = zs[:, None, None]
    return X


def bcs_all(t, prim=None):
    return [BC(t, prim) for _ in range(6)]


# ------------------------------------------------------------ workloads ----

def advection_2d(n=128, seed=2306, steps=200):
    """2D periodic box [0,1]^2, n x n Cartesian cells; rho_inf = 1, p = 1/gamma,
    velocity 2 (cos 30, sin 30) (Mach 2 at 30 deg); seeded Gaussian density
    bump, amplitude 0.1, width 0.1 (minimum-image distance to a centre drawn in
    [0.25, 0.75]^2).  Pressure and velocity uniform: an exact Euler solution
    (pure advection).  MUSCL + minmod, Roe, RK3, CFL 0.5."""
    rng = np.random.default_rng(seed)
    centre = rng.uniform(0.25, 0.75, size=2)
    X = cartesian_nodes(n, n, 1)
    xc = cell_centres(X)
    rho = 1.0 + bump(xc[0], xc[1], centre)
    ang = math.radians(30.0)
    u, v = 2.0 * math.cos(ang), 2.0 * math.sin(ang)
    U0 = conserved(rho, u, v, 0.0, 1.0 / GAMMA)
    return Workload("advection2d", [(n, n, 1)], [X], [U0], [bcs_all(PERIODIC)], limiter="minmod",
                    rk="rk3", cfl=0.5, steps=steps,
                    note=f"bump centre {centre.tolist()}")


def bump(x, y, centre, amp=0.1, width=0.1):
    dx = (x - centre[0] + 0.5) % 1.0 - 0.5
    dy = (y - centre[1] + 0.5) % 1.0 - 0.5
    return amp * np.exp(-(dx * dx + dy * dy) / (width * width))


def ramp_2d(ni=1024, nj=512, ratio=1.02, angle_deg=10.0, steps=500, perturb=0.0, seed=2308):
    """2D supersonic compression ramp (inlet-like): x in [0, 2], 10-deg ramp
    from x = 0.5, top wall y = 1, geometric wall-normal stretching `ratio`;
    the paper's inflow state (Mach 4, 12270 Pa, 217 K) enters at imin and
    fills the domain at t = 0; supersonic outflow (extrapolation) at imax,
    slip wall on the ramp (jmin), freestream at jmax.  MUSCL + van Leer, Roe,
    RK3."""
    X = ramp_nodes(ni, nj, 1, ratio=ratio, angle_deg=angle_deg)
    prim = inlet_inflow()
    U0 = uniform_state((ni, nj, 1), prim, perturb=perturb, seed=seed)
    bcs = [BC(INFLOW, prim), BC(EXTRAPOLATE), BC(SLIP_WALL), BC(INFLOW, prim), BC(PERIODIC), BC(PERIODIC)]
    return Workload("ramp2d", [(ni, nj, 1)], [X], [U0], [bcs], limiter="vanleer", rk="rk3",
                    cfl=0.5, steps=steps)


def periodic_3d(n=256, seed=2307, mach=2.5, limiter="vanleer", steps=100, nj=None, nk=None):
    """3D periodic cube, n^3 cells on the smooth sinusoidal curvilinear map
    (amplitude 5% of the spacing), Mach 2.5 freestream along a seeded unit
    direction, rho and p multiplied by 1 + 0.01 sum_{m=1..5} cos(2 pi k_m.x + psi_m)
    with k_m in {1..4}^3 and psi_m seeded."""
    nj = n if nj is None else nj
    nk = n if nk is None else nk
    rng = np.random.default_rng(seed)
    X = periodic_sine_nodes(n, nj, nk, 0.05, seed=seed + 1)
    d = rng.normal(size=3)
    prim = normalized_freestream(mach, d)
    kvec = rng.integers(1, 5, size=(5, 3))
    psi = rng.uniform(0.0, 2.0 * np.pi, size=5)
    xc = cell_centres(X)
    pert = np.zeros(xc.shape[1:])
    for m in range(5):
        pert += np.cos(2.0 * np.pi * (kvec[m, 0] * xc[0] + kvec[m, 1] * xc[1] + kvec[m, 2] * xc[2]) + psi[m])
    f = 1.0 + 0.01 * pert
    U0 = conserved(prim[0] * f, prim[1], prim[2], prim[3], prim[4] * f)
    return Workload("periodic3d", [(n, nj, nk)], [X], [U0], [bcs_all(PERIODIC)], limiter=limiter,
                    rk="rk3", cfl=0.5, steps=steps)


def ramp_3d(n=512, ratio=1.005, angle_deg=8.0, steps=50, ni=None, nj=None, nk=None, perturb=0.0, seed=2310,
            restrict=1):
    """3D Mach-4 compression ramp, 8-deg ramp extruded in k (periodic in k),
    wall-normal geometric stretching `ratio`, the paper's inflow state.
    restrict = r > 1: the grid of every r-th node of the r-times finer grid
    (e.g. n = 128, restrict = 4: the 128^3 restriction of the 512^3 grid)."""
    ni = n if ni is None else ni
    nj = n if nj is None else nj
    nk = n if nk is None else nk
    X = ramp_nodes(ni, nj, nk, ratio=ratio, angle_deg=angle_deg, depth=1.0, stride=restrict)
    prim = inlet_inflow()
    U0 = uniform_state((ni, nj, nk), prim, perturb=perturb, seed=seed)
    bcs = [BC(INFLOW, prim), BC(EXTRAPOLATE), BC(SLIP_WALL), BC(INFLOW, prim), BC(PERIODIC), BC(PERIODIC)]
    return Workload("ramp3d", [(ni, nj, nk)], [X], [U0], [bcs], limiter="vanleer", rk="rk3",
                    cfl=0.5, steps=steps)


def lattice_3d(sizes=(32, 48, 64, 96, 128), nblk=(4, 4, 4), seed=2309, mach=3.0, ratio=1.01,
               angle_deg=10.0, steps=20, perturb=0.0):
    """Batched multiblock 3D: a global ramp-like curvilinear grid cut into a
    nblk[0] x nblk[1] x nblk[2] lattice; block (a, b, c) has (X_a, Y_b, Z_c)
    cells with X, Y, Z seeded draws from `sizes`.  Faces match point to point
    and exchange two ghost layers.  Mach 3 (paper's p, T) inflow at imin,
    extrapolation at imax, slip wall on the ramp (jmin), freestream at jmax,
    periodic in k."""
    rng = np.random.default_rng(seed)
    Xs = rng.choice(sizes, size=nblk[0]).tolist()
    Ys = rng.choice(sizes, size=nblk[1]).tolist()
    Zs = rng.choice(sizes, size=nblk[2]).tolist()
    NI, NJ, NK = sum(Xs), sum(Ys), sum(Zs)
    Xg = ramp_nodes(NI, NJ, NK, length=2.0, height=1.0, corner=0.5, angle_deg=angle_deg, ratio=ratio,
                    depth=1.0)
    prim = inlet_inflow(mach=mach)
    io = np.concatenate([[0], np.cumsum(Xs)])
    jo = np.concatenate([[0], np.cumsum(Ys)])
    ko = np.concatenate([[0], np.cumsum(Zs)])
    A, B, Cn = nblk
    bid = lambda a, b, c: (c * B + b) * A + a
    dims, nodes, U0, bcs = [], [], [], []
    for c in range(Cn):
        for b in range(B):
            for a in range(A):
                ni, nj, nk = Xs[a], Ys[b], Zs[c]
                dims.append((ni, nj, nk))
                nodes.append(np.ascontiguousarray(
                    Xg[:, ko[c]:ko[c + 1] + 1, jo[b]:jo[b + 1] + 1, io[a]:io[a + 1] + 1]))
                U0.append(uniform_state((ni, nj, nk), prim, perturb=perturb, seed=seed + len(U0)))
                f = [None] * 6
                f[IMIN] = BC(INTERFACE, None, bid(a - 1, b, c), IMAX) if a > 0 else BC(INFLOW, prim)
                f[IMAX] = BC(INTERFACE, None, bid(a + 1, b, c), IMIN) if a < A - 1 else BC(EXTRAPOLATE)
                f[JMIN] = BC(INTERFACE, None, bid(a, b - 1, c), JMAX) if b > 0 else BC(SLIP_WALL)
                f[JMAX] = BC(INTERFACE, None, bid(a, b + 1, c), JMIN) if b < B - 1 else BC(INFLOW, prim)
                f[KMIN] = BC(INTERFACE, None, bid(a, b, (c - 1) % Cn), KMAX)
                f[KMAX] = BC(INTERFACE, None, bid(a, b, (c + 1) % Cn), KMIN)
                if Cn == 1:
                    f[KMIN] = BC(PERIODIC)
                    f[KMAX] = BC(PERIODIC)
                bcs.append(f)
    return Workload("lattice3d", dims, nodes, U0, bcs, limiter="vanleer", rk="rk3", cfl=0.5,
                    steps=steps, note=f"X={Xs} Y={Ys} Z={Zs}")


def restrict_nodes(X, stride):
    """Every `stride`-th node of a grid (the coarse grid of a node restriction)."""
    return np.ascontiguousarray(X[:, ::stride, ::stride, ::stride]) if X.shape[1] > 2 else \
        np.ascontiguousarray(X[:, :, ::stride, ::stride])


def split_i(w, parts):
    """The same grid, state and boundary conditions cut into `parts` blocks
    along i (the 1D decomposition along N_l of the performance model, Sec. 6):
    block p holds i-cells [o_p, o_{p+1}) with o_p = floor(p ni / parts); cut
    faces become block interfaces, an i-periodic pair becomes the interface
    between the last and the first block.  Single-block workloads only."""
    assert len(w.dims) == 1 and 1 <= parts <= w.dims[0][0]
    ni, nj, nk = w.dims[0]
    X, U0, faces = w.nodes[0], w.U0[0], w.bcs[0]
    o = [(p * ni) // parts for p in range(parts + 1)]
    dims, nodes, states, bcs = [], [], [], []
    periodic_i = faces[IMIN].type == PERIODIC
    for p in range(parts):
        dims.append((o[p + 1] - o[p], nj, nk))
        nodes.append(np.ascontiguousarray(X[:, :, :, o[p]:o[p + 1] + 1]))
        states.append(np.ascontiguousarray(U0[:, :, :, o[p]:o[p + 1]]))
        f = list(faces)
        if p > 0:
            f[IMIN] = BC(INTERFACE, None, p - 1, IMAX)
        elif periodic_i and parts > 1:
            f[IMIN] = BC(INTERFACE, None, parts - 1, IMAX)
        if p < parts - 1:
            f[IMAX] = BC(INTERFACE, None, p + 1, IMIN)
        elif periodic_i and parts > 1:
            f[IMAX] = BC(INTERFACE, None, 0, IMIN)
        bcs.append(f)
    return dataclasses.replace(w, name=f"{w.name}/split{parts}", dims=dims, nodes=nodes, U0=states, bcs=bcs,
                               note=(w.note + f" cut into {parts} i-blocks").strip())
