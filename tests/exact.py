"""Closed-form and exact solutions the oracle is pinned against (test-only).

* exact solution of the 1D Riemann problem for the Euler equations of an
  ideal gas (Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics,
  ch. 4: pressure function, Newton iteration for p*, self-similar sampling);
* the theta-beta-Mach relation and the normal-shock jumps across a weak
  oblique shock (NACA Report 1135);
* the Rankine-Hugoniot state behind a stationary normal shock.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


# ------------------------------------------------------------ Riemann ------

def _pressure_fn(p, rho, pk, ck, g):
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pk) / (2.0 * (B + p)))
    else:        # rarefaction
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = (1.0 / (rho * ck)) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_star(left, right, g=1.4, tol=1e-14):
    """(p*, u*) of the exact Riemann solution; left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(tol, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _pressure_fn(p, rl, pl, cl, g)
        fr, dfr = _pressure_fn(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(tol, p - dp)
        if abs(pn - p) < tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _pressure_fn(p, rl, pl, cl, g)
    fr, _ = _pressure_fn(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def riemann_sample(left, right, s, g=1.4):
    """Exact (rho, u, p) at similarity coordinate s = x/t (arrays allowed)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = riemann_star(left, right, g)
    s = np.asarray(s, dtype=np.float64)
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    for n, x in np.ndenumerate(s):
        if x <= us:   # left of the contact
            if ps > pl:   # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if x <= sl:
                    val = (rl, ul, pl)
                else:
                    val = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:         # left rarefaction
                shl = ul - cl
                cml = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - cml
                if x <= shl:
                    val = (rl, ul, pl)
                elif x > stl:
                    val = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - x))
                    val = (rl * (c / cl) ** (2.0 / (g - 1)), 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + x),
                           pl * (c / cl) ** (2 * g / (g - 1)))
        else:         # right of the contact
            if ps > pr:   # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if x >= sr:
                    val = (rr, ur, pr)
                else:
                    val = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:         # right rarefaction
                shr = ur + cr
                cmr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + cmr
                if x >= shr:
                    val = (rr, ur, pr)
                elif x <= str_:
                    val = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - x))
                    val = (rr * (c / cr) ** (2.0 / (g - 1)), 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + x),
                           pr * (c / cr) ** (2 * g / (g - 1)))
        rho[n], u[n], p[n] = val
    return rho, u, p


# ------------------------------------------------------- oblique shocks ----

def theta_of_beta(M, beta, g=1.4):
    """Flow deflection across an oblique shock of wave angle beta."""
    s2 = math.sin(beta) ** 2
    return math.atan(2.0 / math.tan(beta) * (M * M * s2 - 1.0) / (M * M * (g + math.cos(2 * beta)) + 2.0))


def weak_beta(M, theta, g=1.4):
    """Weak-shock wave angle for deflection theta (radians)."""
    mu = math.asin(1.0 / M)
    betas = np.linspace(mu + 1e-9, math.pi / 2 - 1e-9, 20001)
    th = np.array([theta_of_beta(M, b, g) for b in betas])
    bmax = betas[int(np.argmax(th))]
    return brentq(lambda b: theta_of_beta(M, b, g) - theta, mu + 1e-12, bmax)


def oblique_jumps(M, theta, g=1.4):
    """(beta, p2/p1, rho2/rho1, M2) across the weak oblique shock."""
    beta = weak_beta(M, theta, g)
    Mn1 = M * math.sin(beta)
    p21 = 1.0 + 2.0 * g / (g + 1.0) * (Mn1 * Mn1 - 1.0)
    r21 = (g + 1.0) * Mn1 * Mn1 / ((g - 1.0) * Mn1 * Mn1 + 2.0)
    Mn2 = math.sqrt((1.0 + 0.5 * (g - 1.0) * Mn1 * Mn1) / (g * Mn1 * Mn1 - 0.5 * (g - 1.0)))
    M2 = Mn2 / math.sin(beta - theta)
    return beta, p21, r21, M2


def normal_shock_state(rho1, u1, p1, g=1.4):
    """(rho2, u2, p2) behind a stationary normal shock (Rankine-Hugoniot)."""
    c1 = math.sqrt(g * p1 / rho1)
    M1 = u1 / c1
    r21 = (g + 1.0) * M1 * M1 / ((g - 1.0) * M1 * M1 + 2.0)
    p21 = 1.0 + 2.0 * g / (g + 1.0) * (M1 * M1 - 1.0)
    return rho1 * r21, u1 / r21, p1 * p21
