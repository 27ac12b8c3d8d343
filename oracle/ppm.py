"""Test infrastructure: the FP64 oracle of the step with piecewise-parabolic reconstruction (PPM)
on a periodic box or a patch carrying three ghost layers.

Only tests/ import this module; it shares nothing with the CUDA library.

The paper names PPM among the reconstructions of its hydro solvers (Sec. 2) and prints no formula.
The reading here keeps every step of the MUSCL-Hancock/HLLC scheme and replaces only the linear
reconstruction by Colella & Woodward's (1984) parabola, component by component in the primitive
variables q = (rho, u, v, w, p), along each axis d:
  1. monotonised centred slope  dq_i = sign(q_{i+1} - q_{i-1}) min(|q_{i+1} - q_{i-1}|/2,
     2|q_i - q_{i-1}|, 2|q_{i+1} - q_i|) when (q_{i+1} - q_i)(q_i - q_{i-1}) > 0, else 0;
  2. interface value  q_{i+1/2} = q_i + (q_{i+1} - q_i)/2 - (dq_{i+1} - dq_i)/6  (fourth order
     where no slope is limited: (7/12)(q_i + q_{i+1}) - (1/12)(q_{i-1} + q_{i+2}));
  3. edges of cell i: qL = q_{i-1/2}, qR = q_{i+1/2}, then the monotonicity constraints:
     if (qR - q)(q - qL) <= 0 both edges become q (a local extremum is flattened); otherwise, with
     D = qR - qL and Q6 = 6 (q - (qL + qR)/2): if D Q6 > D^2, qL = 3q - 2qR; else if -D^2 > D Q6,
     qR = 3q - 2qL (the parabola then has no extremum inside the cell);
  4. Hancock predictor with the parabola's centre slope D = qR - qL in place of the PLM slope:
     q_h = q - dt/(2 dx) ((A_x(q) D_x + A_y(q) D_y) + A_z(q) D_z);
  5. face states at time n+1/2: q_h + (qR - q) on the low side of a face, q_h + (qL - q) on the
     high side (with PLM edges q +- dq/2 these are the usual q_h +- dq/2), floored as in the PLM
     step; HLLC flux; conservative update as in the PLM step.
No characteristic tracing and no flattening near shocks are applied (the predictor is the same
unsplit primitive Hancock step as with PLM).  The stencil radius is 3 cells.
"""
import numpy as np

from . import config as _config
from . import hllc_n, recover


def _sh(a, s, axis):
    """a_{i+s} along the array axis, periodic."""
    return np.roll(a, -s, axis=axis)


def mc_slope(q, axis):
    dl = q - _sh(q, -1, axis)
    dr = _sh(q, 1, axis) - q
    dc = 0.5 * (_sh(q, 1, axis) - _sh(q, -1, axis))
    lim = np.minimum(np.abs(dc), np.minimum(2.0 * np.abs(dl), 2.0 * np.abs(dr)))
    return np.where(dl * dr > 0.0, np.copysign(lim, dc), 0.0)


def interfaces(q, axis):
    """q_{i+1/2} of every cell i along the axis (step 2)."""
    dq = mc_slope(q, axis)
    return q + 0.5 * (_sh(q, 1, axis) - q) - (_sh(dq, 1, axis) - dq) / 6.0


def ppm_edges(q, axis, limiter=None):
    """(qL, qR) of every cell along the axis after the monotonicity constraints (steps 2-3)."""
    qR = interfaces(q, axis)
    qL = _sh(qR, -1, axis)
    ext = (qR - q) * (q - qL) <= 0.0
    D = qR - qL
    Q6 = 6.0 * (q - 0.5 * (qL + qR))
    lo = ~ext & (D * Q6 > D * D)
    hi = ~ext & ~lo & (-(D * D) > D * Q6)
    nL = np.where(ext, q, np.where(lo, 3.0 * q - 2.0 * qR, qL))
    nR = np.where(ext, q, np.where(hi, 3.0 * q - 2.0 * qL, qR))
    return nL, nR


def plm_edges(q, axis, limiter="minmod"):
    """(q - dq/2, q + dq/2) with the PLM limited slope: the PLM step written in edge form."""
    a = q - _sh(q, -1, axis)
    b = _sh(q, 1, axis) - q
    if limiter == "minmod":
        dq = np.where(a * b <= 0.0, 0.0, np.where(np.abs(a) <= np.abs(b), a, b))
    elif limiter == "none":
        dq = 0.5 * (a + b)
    else:
        raise ValueError(limiter)
    return q - 0.5 * dq, q + 0.5 * dq


def hancock_term(q, D, d, gamma):
    """A_d(q) D: the primitive-variable Jacobian of direction d applied to D."""
    n = 1 + d
    un = q[n]
    out = np.empty_like(q)
    out[0] = un * D[0] + q[0] * D[n]
    out[1] = un * D[1]
    out[2] = un * D[2]
    out[3] = un * D[3]
    out[n] = out[n] + D[4] / q[0]
    out[4] = gamma * q[4] * D[n] + un * D[4]
    return out


GHOST = 3


def step_patch(Ug, dx, dt, cfg=None):
    """One step of a patch carrying three ghost layers, Ug (5, nz+6, ny+6, nx+6) -> interior
    (5, nz, ny, nx).  The periodic step of the ghosted box is exact on the interior: the wrap only
    reaches cells within three of the box's faces, which no interior update reads."""
    return step_periodic(Ug, dx, dt, cfg)[:, GHOST:-GHOST, GHOST:-GHOST, GHOST:-GHOST]


def step_periodic(U, dx, dt, cfg=None, edges=ppm_edges, limiter=None):
    """One step of the periodic box U (5, nz, ny, nx) with the reconstruction `edges`."""
    cfg = cfg or _config()
    U = np.asarray(U, dtype=np.float64)
    q = recover(U, cfg)
    axes = (3, 2, 1)  # array axis of x, y, z
    E = [edges(q, axes[d], limiter) for d in range(3)]
    t = [hancock_term(q, E[d][1] - E[d][0], d, cfg.gamma) for d in range(3)]
    qh = q - (0.5 * dt / dx) * ((t[0] + t[1]) + t[2])
    div = None
    for d in range(3):
        ax = axes[d]
        qL = qh + (E[d][1] - q)                   # low side of face i+1/2: cell i's high edge
        qR = _sh(qh + (E[d][0] - q), 1, ax)       # high side: cell i+1's low edge
        for s in (qL, qR):
            s[0] = np.maximum(s[0], cfg.rho_floor)
            s[4] = np.maximum(s[4], cfg.p_floor)
        F = hllc_n(qL, qR, d, cfg)                # flux through face i+1/2
        dF = F - _sh(F, -1, ax)
        div = dF if div is None else div + dF
    return U - (dt / dx) * div
