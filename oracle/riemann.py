"""Exact solution of the Riemann problem for the 1D Euler equations (ideal gas).

TEST INFRASTRUCTURE ONLY (part of the oracle).  Written from the mathematics:
the star-region pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is
the shock (Rankine-Hugoniot) branch for p > p_K and the isentropic rarefaction
branch for p <= p_K; the self-similar solution is then sampled at x/t.  This
is the textbook pressure-function method for the exact Riemann solver; it pins
the oracle's shock-tube runs (Sod and Lax tubes of the Euler-equation section
of the paper, and random tubes), since those have a closed-form solution.
"""
from __future__ import annotations

import numpy as np


def _f_and_df(p, rho, pk, c, g):
    if p > pk:  # shock branch
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = np.sqrt(A / (p + B))
        f = (p - pk) * q
        df = q * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction branch
        r = p / pk
        f = 2.0 * c / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * c) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, gamma=1.4, tol=1e-14, max_iter=200):
    """left/right = (rho, u, p).  Returns (p_star, u_star)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl = np.sqrt(g * pl / rl)
    cr = np.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated; no star region")
    # two-rarefaction guess, then Newton on the pressure function
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl**z + cr / pr**z)) ** (1.0 / z)
    p = max(p, 1e-14)
    for _ in range(max_iter):
        fl, dfl = _f_and_df(p, rl, pl, cl, g)
        fr, dfr = _f_and_df(p, rr, pr, cr, g)
        p_new = p - (fl + fr + ur - ul) / (dfl + dfr)
        if p_new < 0.0:
            p_new = 0.5 * p
        if abs(p_new - p) <= tol * 0.5 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f_and_df(p, rl, pl, cl, g)
    fr, _ = _f_and_df(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, gamma=1.4):
    """Primitive (rho, u, p) of the exact solution at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    ps, us = star_state(left, right, gamma)
    cl = np.sqrt(g * pl / rl)
    cr = np.sqrt(g * pr / rr)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for idx, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * np.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= sl:
                    rho[idx], u[idx], p[idx] = rl, ul, pl
                else:
                    rho[idx] = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                    u[idx], p[idx] = us, ps
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                head, tail = ul - cl, us - csl
                if s <= head:
                    rho[idx], u[idx], p[idx] = rl, ul, pl
                elif s >= tail:
                    rho[idx] = rl * (ps / pl) ** (1.0 / g)
                    u[idx], p[idx] = us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    u[idx] = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    rho[idx] = rl * (c / cl) ** (2.0 / (g - 1.0))
                    p[idx] = pl * (c / cl) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= sr:
                    rho[idx], u[idx], p[idx] = rr, ur, pr
                else:
                    rho[idx] = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                    u[idx], p[idx] = us, ps
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                head, tail = ur + cr, us + csr
                if s >= head:
                    rho[idx], u[idx], p[idx] = rr, ur, pr
                elif s <= tail:
                    rho[idx] = rr * (ps / pr) ** (1.0 / g)
                    u[idx], p[idx] = us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    u[idx] = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    rho[idx] = rr * (c / cr) ** (2.0 / (g - 1.0))
                    p[idx] = pr * (c / cr) ** (2.0 * g / (g - 1.0))
    return rho, u, p


def wave_speeds(left, right, gamma=1.4):
    """Fastest left- and right-going signal speeds (for domain-of-influence checks)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    ps, us = star_state(left, right, gamma)
    cl = np.sqrt(g * pl / rl)
    cr = np.sqrt(g * pr / rr)
    if ps > pl:
        smin = ul - cl * np.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
    else:
        smin = ul - cl
    if ps > pr:
        smax = ur + cr * np.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
    else:
        smax = ur + cr
    return smin, smax
