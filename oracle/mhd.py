"""Test infrastructure: the FP64 oracle of one step of ideal MHD with hyperbolic divergence
cleaning on a periodic box or a patch carrying two ghost layers.

Only tests/ import this module; it shares nothing with the CUDA library.

The paper's second code runs magnetohydrodynamics on the GPU (Enzo MHD, Sec. 4) and prints no
equations.  The readings here (each a textbook choice):
  - Ideal MHD in units where the magnetic pressure is |B|^2/2; conserved state
    U = (rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi), E = p/(gamma-1) + |m|^2/(2 rho) + |B|^2/2;
    psi the GLM cleaning scalar of Dedner et al. (2002): the normal field's flux is psi and psi's
    flux is c_h^2 B_n, and psi decays by the factor exp(-alpha c_h dt / dx) after each step.
  - c_h = (cfl / 3) dx / dt, the largest speed the unsplit time step allows on each axis (the CFL
    sum runs over three axes), and alpha = 0.4.
  - Primitive variables w = (rho, u, v, w, p, B_x, B_y, B_z, psi) reconstructed component by
    component with the PLM limiter of the hydro step (MinMod, MC or none).
  - Hancock predictor in conservative form (Toro, Sec. 14.4, the unsplit version): each cell's six
    extrapolated states w +- dw_d / 2, as conserved states, advanced by half a step with the flux
    differences of the cell's own extrapolated states along every axis,
    U_face^{n+1/2} = U_face - dt/(2 dx) sum_d (F_d(U_{d,+}) - F_d(U_{d,-})),
    then recovered and floored (rho, p) as in the hydro step.
  - HLL flux (Harten, Lax & van Leer) between the face states with Davis speed bounds from the fast
    magnetosonic speed c_f^2 = ((a^2 + b^2) + sqrt((a^2 + b^2)^2 - 4 a^2 b_n^2)) / 2,
    a^2 = gamma p / rho, b^2 = |B|^2 / rho, b_n^2 = B_n^2 / rho; before it, the normal field and psi
    at the face take the solution of the 2x2 cleaning system:
    B_n* = (B_nL + B_nR)/2 - (psi_R - psi_L)/(2 c_h),  psi* = (psi_L + psi_R)/2 - c_h (B_nR - B_nL)/2,
    B_n* replaces B_n in both states, and the B_n and psi fluxes are psi* and c_h^2 B_n*.
  - Update U^{n+1} = U^n - dt/dx ((dF_x + dF_y) + dF_z); then the psi damping.
  - CFL dt = cfl dx / max_cells sum_d (|u_d| + c_f,d).
"""
import numpy as np

from . import config as _config

NV = 9
ALPHA = 0.4


def _sh(a, s, axis):
    return np.roll(a, -s, axis=axis)


def slope(a, b, limiter):
    """The PLM limited slope of left and right differences a, b (as in the hydro step)."""
    if limiter == "none":
        return 0.5 * (a + b)
    if limiter == "minmod":
        return np.where(a * b <= 0.0, 0.0, np.where(np.abs(a) <= np.abs(b), a, b))
    if limiter == "mc":
        ta, tb, m = 2.0 * a, 2.0 * b, 0.5 * (a + b)
        best = np.where(np.abs(tb) < np.abs(ta), tb, ta)
        best = np.where(np.abs(m) < np.abs(best), m, best)
        return np.where(a * b <= 0.0, 0.0, best)
    raise ValueError(limiter)


def recover(U, cfg):
    """Primitive state w of conserved U, rho and p floored (rho before dividing, p after)."""
    rho = np.maximum(U[0], cfg.rho_floor)
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    kin = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho
    mag = 0.5 * (U[5] * U[5] + U[6] * U[6] + U[7] * U[7])
    p = np.maximum((cfg.gamma - 1.0) * ((U[4] - kin) - mag), cfg.p_floor)
    return np.stack([rho, u, v, w, p, U[5], U[6], U[7], U[8]])


def conserved(q, cfg):
    rho = q[0]
    kin = 0.5 * rho * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3])
    mag = 0.5 * (q[5] * q[5] + q[6] * q[6] + q[7] * q[7])
    E = q[4] / (cfg.gamma - 1.0) + kin + mag
    return np.stack([rho, rho * q[1], rho * q[2], rho * q[3], E, q[5], q[6], q[7], q[8]])


def flux(q, d, ch, cfg):
    """Physical flux along axis d (0, 1, 2) of primitive state q, with the GLM terms."""
    n = 1 + d
    rho, p = q[0], q[4]
    un, Bn = q[n], q[5 + d]
    B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7]
    pt = p + 0.5 * B2
    uB = q[1] * q[5] + q[2] * q[6] + q[3] * q[7]
    E = p / (cfg.gamma - 1.0) + 0.5 * rho * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) + 0.5 * B2
    F = np.empty_like(q)
    F[0] = rho * un
    for k in range(3):
        F[1 + k] = rho * un * q[1 + k] - Bn * q[5 + k]
    F[n] = F[n] + pt
    F[4] = (E + pt) * un - Bn * uB
    for k in range(3):
        F[5 + k] = un * q[5 + k] - q[1 + k] * Bn
    F[5 + d] = q[8]                 # the normal field's flux is psi
    F[8] = ch * ch * Bn              # psi's flux
    return F


def fast_speed(q, d, cfg):
    rho = q[0]
    a2 = cfg.gamma * q[4] / rho
    b2 = (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]) / rho
    bn2 = q[5 + d] * q[5 + d] / rho
    s = a2 + b2
    return np.sqrt(0.5 * (s + np.sqrt(np.maximum(s * s - 4.0 * a2 * bn2, 0.0))))


def glm_face(BnL, BnR, psiL, psiR, ch):
    """Solution of the 2x2 cleaning system at the face: (B_n*, psi*)."""
    Bm = 0.5 * (BnL + BnR) - (psiR - psiL) / (2.0 * ch)
    pm = 0.5 * (psiL + psiR) - 0.5 * ch * (BnR - BnL)
    return Bm, pm


def hll(qL, qR, d, ch, cfg):
    """HLL flux along axis d between primitive states qL, qR (after the GLM face solution)."""
    Bm, pm = glm_face(qL[5 + d], qR[5 + d], qL[8], qR[8], ch)
    qL = qL.copy()
    qR = qR.copy()
    qL[5 + d] = Bm
    qR[5 + d] = Bm
    qL[8] = pm
    qR[8] = pm
    n = 1 + d
    cL, cR = fast_speed(qL, d, cfg), fast_speed(qR, d, cfg)
    SL = np.minimum(qL[n] - cL, qR[n] - cR)
    SR = np.maximum(qL[n] + cL, qR[n] + cR)
    FL, FR = flux(qL, d, ch, cfg), flux(qR, d, ch, cfg)
    UL, UR = conserved(qL, cfg), conserved(qR, cfg)
    Fs = (SR * FL - SL * FR + SL * SR * (UR - UL)) / (SR - SL)
    F = np.where(SL >= 0.0, FL, np.where(SR <= 0.0, FR, Fs))
    F[5 + d] = pm                    # the GLM pair is exact: psi* and c_h^2 B_n*
    F[8] = ch * ch * Bm
    return F


def floor_state(q, cfg):
    q = q.copy()
    q[0] = np.maximum(q[0], cfg.rho_floor)
    q[4] = np.maximum(q[4], cfg.p_floor)
    return q


def ch_of(dx, dt, cfg):
    return (cfg.cfl / 3.0) * dx / dt


def step_periodic(U, dx, dt, cfg=None, limiter="minmod"):
    """One step of the periodic box U (9, nz, ny, nx) -> U^{n+1}."""
    cfg = cfg or _config()
    U = np.asarray(U, dtype=np.float64)
    ch = ch_of(dx, dt, cfg)
    q = recover(U, cfg)
    axes = (3, 2, 1)
    lo, hi = [], []
    for d in range(3):
        ax = axes[d]
        dq = slope(q - _sh(q, -1, ax), _sh(q, 1, ax) - q, limiter)
        lo.append(q - 0.5 * dq)
        hi.append(q + 0.5 * dq)
    # conservative Hancock predictor: sum over axes of the flux difference of the cell's own states
    dF = None
    for d in range(3):
        t = flux(hi[d], d, ch, cfg) - flux(lo[d], d, ch, cfg)
        dF = t if dF is None else dF + t
    h = 0.5 * dt / dx
    face_lo = [floor_state(recover(conserved(lo[d], cfg) - h * dF, cfg), cfg) for d in range(3)]
    face_hi = [floor_state(recover(conserved(hi[d], cfg) - h * dF, cfg), cfg) for d in range(3)]
    div = None
    for d in range(3):
        ax = axes[d]
        F = hll(face_hi[d], _sh(face_lo[d], 1, ax), d, ch, cfg)   # face i+1/2
        t = F - _sh(F, -1, ax)
        div = t if div is None else div + t
    out = U - (dt / dx) * div
    out[8] = out[8] * np.exp(-ALPHA * ch * dt / dx)
    return out


GHOST = 2


def step_patch(Ug, dx, dt, cfg=None, limiter="minmod"):
    """One step of a patch carrying two ghost layers, Ug (9, nz+4, ny+4, nx+4) -> interior
    (9, nz, ny, nx).  The periodic step of the ghosted box is exact on the interior: the wrap only
    reaches cells within two of the box's faces, which no interior update reads."""
    return step_periodic(Ug, dx, dt, cfg, limiter)[:, GHOST:-GHOST, GHOST:-GHOST, GHOST:-GHOST]


def cfl_patch(Ug, dx, cfg=None):
    """CFL dt of the interior of a patch carrying two ghost layers."""
    return cfl_periodic(np.asarray(Ug)[:, GHOST:-GHOST, GHOST:-GHOST, GHOST:-GHOST], dx, cfg)


def cfl_periodic(U, dx, cfg=None):
    cfg = cfg or _config()
    q = recover(np.asarray(U, dtype=np.float64), cfg)
    s = ((np.abs(q[1]) + fast_speed(q, 0, cfg)) + (np.abs(q[2]) + fast_speed(q, 1, cfg))) + \
        (np.abs(q[3]) + fast_speed(q, 2, cfg))
    return cfg.cfl * (dx / s.max())


def div_b(U, dx):
    """Central-difference divergence of B on the periodic box."""
    return ((_sh(U[5], 1, 2) - _sh(U[5], -1, 2)) + (_sh(U[6], 1, 1) - _sh(U[6], -1, 1)) +
            (_sh(U[7], 1, 0) - _sh(U[7], -1, 0))) / (2.0 * dx)
