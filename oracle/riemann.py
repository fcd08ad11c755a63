"""Exact solution of the Riemann problem of the 1D Euler equations, ideal gas.

TEST INFRASTRUCTURE ONLY (pins the oracle's Sod shock tube, the 1D Euler
configuration with gamma = 1.4). This is the textbook construction (Toro,
"Riemann Solvers and Numerical Methods for Fluid Dynamics", Ch. 4): the star
pressure p* is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
shock (Rankine-Hugoniot) branch for p > p_K and the isentropic rarefaction
branch otherwise; u* follows from the same functions, and the solution is
sampled on the similarity variable x/t.
"""
import math

import numpy as np


def _fk(p, rk, pk, ck, g):
    if p > pk:  # shock
        a = 2.0 / ((g + 1.0) * rk)
        b = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(a / (p + b))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + b))
    # rarefaction
    pr = p / pk
    f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rk * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, g):
    """(p*, u*) by Newton iteration on the pressure function."""
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    # two-rarefaction initial guess
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, cl, g)
        fr, dr = _fk(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        if pn < 0:
            pn = 1e-12
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(rl, ul, pl, rr, ur, pr, g, xi):
    """Primitive (rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    ps, us = star_state(rl, ul, pl, rr, ur, pr, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for i, s in enumerate(xi.ravel()):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= sl:
                    r, v, q = rl, ul, pl
                else:
                    r, v, q = rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
            else:  # left rarefaction
                head = ul - cl
                csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                tail = us - csl
                if s <= head:
                    r, v, q = rl, ul, pl
                elif s >= tail:
                    r, v, q = rl * (ps / pl) ** (1.0 / g), us, ps
                else:
                    v = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    q = pl * (c / cl) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= sr:
                    r, v, q = rr, ur, pr
                else:
                    r, v, q = rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
            else:  # right rarefaction
                head = ur + cr
                csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                tail = us + csr
                if s >= head:
                    r, v, q = rr, ur, pr
                elif s <= tail:
                    r, v, q = rr * (ps / pr) ** (1.0 / g), us, ps
                else:
                    v = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    q = pr * (c / cr) ** (2.0 * g / (g - 1.0))
        rho.flat[i], u.flat[i], p.flat[i] = r, v, q
    return rho, u, p
