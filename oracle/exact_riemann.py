"""Exact solution of the 1D Riemann problem for an ideal gas (TEST INFRASTRUCTURE).

Used to pin the oracle on the Sod shock tube of Sec. 5.1 (the paper checks its
solver against "the known analytic solution").  Written from the textbook
construction (E. F. Toro, Riemann Solvers and Numerical Methods for Fluid
Dynamics, ch. 4): the star pressure is the root of
f(p) = f_L(p) + f_R(p) + (u_R - u_L), each f_K the shock (Rankine-Hugoniot) or
rarefaction (isentropic) branch, found by Newton iteration; the solution is then
sampled along x/t.  Pinned itself by the published star values of Toro's test 1
(tests/golden/toro_test1.txt), and by the integral conservation laws and the
Rankine-Hugoniot speeds of its sampled solution.
"""
from __future__ import annotations

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        Bk = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * np.sqrt(A / (p + Bk))
        df = np.sqrt(A / (Bk + p)) * (1.0 - (p - pk) / (2.0 * (Bk + p)))
    else:  # rarefaction
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, gamma=1.4, tol=1e-14, maxit=100):
    """(p*, u*) for left/right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    # two-rarefaction guess, a standard positive starting value
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, tol)
    for _ in range(maxit):
        fl, dfl = _fk(p, rl, pl, cl, g)
        fr, dfr = _fk(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, tol)
        if abs(pn - p) / (0.5 * (pn + p)) < tol:
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, gamma=1.4):
    """Primitive (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    ps, us = star_state(left, right, g)
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((3, xi.size))
    gm = (g - 1.0) / (g + 1.0)
    for n, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * ((ps / pl + gm) / (gm * ps / pl + 1.0))
                S = ul - cl * np.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                st = (rl, ul, pl) if s <= S else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                sh, stl = ul - cl, us - cs
                if s <= sh:
                    st = (rl, ul, pl)
                elif s >= stl:
                    st = (rs, us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * (ul - s))
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    st = (r, u, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rs = rr * ((ps / pr + gm) / (gm * ps / pr + 1.0))
                S = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                st = (rr, ur, pr) if s >= S else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                sh, stt = ur + cr, us + cs
                if s >= sh:
                    st = (rr, ur, pr)
                elif s <= stt:
                    st = (rs, us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2.0 * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - (g - 1.0) / 2.0 * (ur - s))
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    st = (r, u, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        out[:, n] = st
    return out


def cell_average_density(left, right, x0, t, edges, gamma=1.4, nsub=64):
    """Cell averages of rho over the cells [edges[i], edges[i+1]] at time t."""
    edges = np.asarray(edges, dtype=np.float64)
    out = np.zeros(edges.size - 1)
    for i in range(edges.size - 1):
        xs = edges[i] + (np.arange(nsub) + 0.5) / nsub * (edges[i + 1] - edges[i])
        out[i] = sample(left, right, (xs - x0) / t, gamma)[0].mean()
    return out
