"""Test infrastructure: exact solution of the 1D Riemann problem of the ideal-gas Euler equations.

Used to pin the HLLC/MUSCL-Hancock oracle on shock tubes.  The method is the classical one
(Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", Ch. 4): the star pressure p*
is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-Hugoniot) or
rarefaction (isentropic) relation across the K wave; u* follows from p*, and the self-similar
solution is sampled at x/t.  Written from the mathematics; plain Python scalars.
"""
import math

import numpy as np


def _f_and_df(p, rho, pk, ck, g):
    """Velocity jump across the wave of one side for star pressure p, and its derivative."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    e = (g - 1.0) / (2.0 * g)
    r = (p / pk) ** e
    return 2.0 * ck / (g - 1.0) * (r - 1.0), 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(left, right, gamma):
    """(p*, u*) of the Riemann problem with left/right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    du = ur - ul
    if 2.0 * (cl + cr) / (g - 1.0) <= du:
        raise ValueError("initial data generate vacuum")
    # Start from the two-rarefaction guess, which is exact when both waves are rarefactions.
    e = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * du) / (cl / pl ** e + cr / pr ** e)) ** (1.0 / e)
    p = max(p, 1e-14)
    for _ in range(100):
        fl, dfl = _f_and_df(p, rl, pl, cl, g)
        fr, dfr = _f_and_df(p, rr, pr, cr, g)
        pn = p - (fl + fr + du) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= 1e-14 * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, cl, g)
    fr, _ = _f_and_df(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, gamma, xi):
    """Primitive state (rho, u, p) at similarity coordinates xi = (x - x0)/t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    ps, us = star_state(left, right, gamma)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.zeros((3,) + xi.shape)
    gm = (g - 1.0) / (g + 1.0)
    for idx, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                if s <= sl:
                    st = (rl, ul, pl)
                else:
                    st = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                shl, stl = ul - cl, us - csl
                if s <= shl:
                    st = (rl, ul, pl)
                elif s >= stl:
                    st = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    r = rl * (c / cl) ** (2.0 / (g - 1.0))
                    st = (r, u, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                if s >= sr:
                    st = (rr, ur, pr)
                else:
                    st = (rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps)
            else:  # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                shr, str_ = ur + cr, us + csr
                if s >= shr:
                    st = (rr, ur, pr)
                elif s <= str_:
                    st = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    r = rr * (c / cr) ** (2.0 / (g - 1.0))
                    st = (r, u, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        out[(slice(None),) + idx] = st
    return out
