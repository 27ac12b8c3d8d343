"""Test infrastructure: the plain FP64 CPU oracle of the MUSCL-Hancock/HLLC hydro step.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg import this package.
It shares no code with the CUDA library (``paper_1412_0934_gb300``) and never imports it.

The scheme follows the paper's description of the hydro path (Sec. 2: the ideal-fluid Euler
equations solved with PLM, Colella & Glaz 1985; Sec. 4: every flux that updates a patch's cells
plus the adaptive time step) with the textbook steps written out in ``euler_oracle.hpp``.
Arrays are numpy float64 of shape (5, nz, ny, nx) -- fields (rho, m_x, m_y, m_z, E), x fastest
-- or (5, nz+4, ny+4, nx+4) for patches carrying 2 ghost layers.
"""
import ctypes
import os

import numpy as np

from . import build as _build

GHOST = 2

_lib = None


class OracleConfig(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("rho_floor", ctypes.c_double),
                ("p_floor", ctypes.c_double), ("limiter", ctypes.c_int)]


LIMITERS = {"minmod": 0, "mc": 1, "none": 2}


def config(gamma=5.0 / 3.0, cfl=0.8, rho_floor=1e-10, p_floor=1e-14, limiter="minmod"):
    lim = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
    return OracleConfig(gamma, cfl, rho_floor, p_floor, lim)


def load(so):
    """A ctypes handle on an oracle library built from these sources, argument types set."""
    L = ctypes.CDLL(so)
    P = ctypes.POINTER(OracleConfig)
    d = ctypes.c_double
    i = ctypes.c_int
    vp = ctypes.c_void_p
    L.oracle_step_periodic.argtypes = [P, vp, vp, i, i, i, d, d]
    L.oracle_step_patch.argtypes = [P, vp, vp, i, i, i, d, d]
    L.oracle_cfl_periodic.argtypes = [P, vp, i, i, i, d]
    L.oracle_cfl_periodic.restype = d
    L.oracle_cfl_patch.argtypes = [P, vp, i, i, i, d]
    L.oracle_cfl_patch.restype = d
    L.oracle_step_periodic_tangent.argtypes = [P, vp, vp, vp, vp, i, i, i, d, d]
    L.oracle_step_periodic_adjoint.argtypes = [P, vp, vp, vp, i, i, i, d, d, i]
    L.oracle_step_patch_adjoint.argtypes = [P, vp, vp, vp, i, i, i, d, d]
    L.oracle_hllc.argtypes = [P, vp, vp, i, vp]
    L.oracle_hllc_n.argtypes = [P, vp, vp, i, vp, ctypes.c_long]
    L.oracle_recover.argtypes = [P, vp, vp, ctypes.c_long]
    L.oracle_prim_to_cons.argtypes = [P, vp, vp, ctypes.c_long]
    L.oracle_prim_to_cons_adjoint.argtypes = [P, vp, vp, vp, ctypes.c_long]
    L.oracle_count_ops.argtypes = [P, vp, i, i, i, d, d, vp]
    L.oracle_patch_boundary_fluxes.argtypes = [P, vp, i, i, i, d, d, vp]
    L.oracle_threads.argtypes = []
    L.oracle_threads.restype = i
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def threads():
    """OpenMP threads of the oracle's parallel stages on this host."""
    return int(lib().oracle_threads())


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data


def _check(rc):
    if rc != 0:
        raise ValueError("oracle call rejected its arguments")


def step_periodic(U, dx, dt, cfg=None):
    """One step of the periodic box U (5, nz, ny, nx) -> U^{n+1}."""
    cfg = cfg or config()
    U, pu = _c(U)
    _, nz, ny, nx = U.shape
    out = np.empty_like(U)
    _check(lib().oracle_step_periodic(ctypes.byref(cfg), pu, out.ctypes.data, nx, ny, nz, dx, dt))
    return out


def step_patch(Ug, dx, dt, cfg=None):
    """One step of a ghosted patch Ug (5, nz+4, ny+4, nx+4) -> interior U^{n+1} (5, nz, ny, nx)."""
    cfg = cfg or config()
    Ug, pu = _c(Ug)
    _, NZ, NY, NX = Ug.shape
    nx, ny, nz = NX - 2 * GHOST, NY - 2 * GHOST, NZ - 2 * GHOST
    out = np.empty((5, nz, ny, nx))
    _check(lib().oracle_step_patch(ctypes.byref(cfg), pu, out.ctypes.data, nx, ny, nz, dx, dt))
    return out


def patch_boundary_fluxes(Ug, dx, dt, cfg=None):
    """Fluxes through the six boundary faces of the ghosted patch Ug's interior, as step_patch
    applies them: (5, R) with R = 2 (ny nz + nx nz + nx ny), per field x-low [nz][ny], x-high,
    y-low [nz][nx], y-high, z-low [ny][nx], z-high."""
    cfg = cfg or config()
    Ug, pu = _c(Ug)
    _, NZ, NY, NX = Ug.shape
    nx, ny, nz = NX - 2 * GHOST, NY - 2 * GHOST, NZ - 2 * GHOST
    out = np.empty((5, 2 * (ny * nz + nx * nz + nx * ny)))
    _check(lib().oracle_patch_boundary_fluxes(ctypes.byref(cfg), pu, nx, ny, nz, dx, dt, out.ctypes.data))
    return out


def cfl_periodic(U, dx, cfg=None):
    cfg = cfg or config()
    U, pu = _c(U)
    _, nz, ny, nx = U.shape
    return lib().oracle_cfl_periodic(ctypes.byref(cfg), pu, nx, ny, nz, dx)


def cfl_patch(Ug, dx, cfg=None):
    cfg = cfg or config()
    Ug, pu = _c(Ug)
    _, NZ, NY, NX = Ug.shape
    return lib().oracle_cfl_patch(ctypes.byref(cfg), pu, NX - 4, NY - 4, NZ - 4, dx)


def step_periodic_tangent(U, dU, dx, dt, cfg=None):
    """(U^{n+1}, J dU) of one periodic step, by dual numbers."""
    cfg = cfg or config()
    U, pu = _c(U)
    dU, pd = _c(dU)
    _, nz, ny, nx = U.shape
    out = np.empty_like(U)
    dout = np.empty_like(U)
    _check(lib().oracle_step_periodic_tangent(ctypes.byref(cfg), pu, pd, out.ctypes.data, dout.ctypes.data,
                                              nx, ny, nz, dx, dt))
    return out, dout


def step_periodic_adjoint(U, lam_out, dx, dt, cfg=None, block=8):
    """J^T lam_out of one periodic step (dt held fixed), by a reverse-mode tape."""
    cfg = cfg or config()
    U, pu = _c(U)
    L, pl = _c(lam_out)
    _, nz, ny, nx = U.shape
    lam_in = np.empty_like(U)
    _check(lib().oracle_step_periodic_adjoint(ctypes.byref(cfg), pu, pl, lam_in.ctypes.data, nx, ny, nz, dx, dt,
                                              block))
    return lam_in


def step_patch_adjoint(Ug, lam_out, dx, dt, cfg=None):
    """J^T lam_out of one ghosted-patch step; result on the ghosted box."""
    cfg = cfg or config()
    Ug, pu = _c(Ug)
    L, pl = _c(lam_out)
    _, NZ, NY, NX = Ug.shape
    lam_in = np.empty_like(Ug)
    _check(lib().oracle_step_patch_adjoint(ctypes.byref(cfg), pu, pl, lam_in.ctypes.data, NX - 4, NY - 4, NZ - 4,
                                           dx, dt))
    return lam_in


def hllc(qL, qR, d, cfg=None):
    cfg = cfg or config()
    qL, pl = _c(qL)
    qR, pr = _c(qR)
    F = np.empty(5)
    _check(lib().oracle_hllc(ctypes.byref(cfg), pl, pr, d, F.ctypes.data))
    return F


def hllc_n(qL, qR, d, cfg=None):
    """HLLC fluxes (5, ...) of the faces of normal d between primitive states qL, qR (5, ...)."""
    cfg = cfg or config()
    qL, pl = _c(qL)
    qR, pr = _c(qR)
    F = np.empty_like(qL)
    _check(lib().oracle_hllc_n(ctypes.byref(cfg), pl, pr, d, F.ctypes.data, qL[0].size))
    return F


def recover(U, cfg=None):
    """Primitive state (5, ...) of conserved state U (5, ...)."""
    cfg = cfg or config()
    U, pu = _c(U)
    n = U[0].size
    q = np.empty_like(U)
    _check(lib().oracle_recover(ctypes.byref(cfg), pu, q.ctypes.data, n))
    return q


def prim_to_cons(q, cfg=None):
    cfg = cfg or config()
    q, pq = _c(q)
    n = q[0].size
    U = np.empty_like(q)
    _check(lib().oracle_prim_to_cons(ctypes.byref(cfg), pq, U.ctypes.data, n))
    return U


def prim_to_cons_adjoint(q, lamU, cfg=None):
    cfg = cfg or config()
    q, pq = _c(q)
    L, pl = _c(lamU)
    n = q[0].size
    lamq = np.empty_like(q)
    _check(lib().oracle_prim_to_cons_adjoint(ctypes.byref(cfg), pq, pl, lamq.ctypes.data, n))
    return lamq


def count_ops(U, dx, dt, cfg=None):
    """Arithmetic operations (+ - * / sqrt) per unit of each stage of one periodic step:
    dict(recover per cell, slopes per cell, predict per cell, face per face, update per cell,
    per_cell = recover + slopes + predict + 3 * face + update)."""
    cfg = cfg or config()
    U, pu = _c(U)
    _, nz, ny, nx = U.shape
    out = np.zeros(25)
    _check(lib().oracle_count_ops(ctypes.byref(cfg), pu, nx, ny, nz, dx, dt, out.ctypes.data))
    d = dict(recover=out[0], slopes=out[1], predict=out[2], face=out[3], update=out[4])
    d["per_cell"] = out[0] + out[1] + out[2] + 3 * out[3] + out[4]
    mult = [1, 1, 1, 3, 1]
    kinds = ("addsub", "mul", "div", "sqrt")
    d["by_kind"] = {k: float(sum(mult[s] * out[5 + 4 * s + i] for s in range(5))) for i, k in enumerate(kinds)}
    return d


def fill_ghosts_periodic(U):
    """Ghosted (5, nz+4, ny+4, nx+4) copy of the periodic box U."""
    return np.pad(U, ((0, 0), (GHOST, GHOST), (GHOST, GHOST), (GHOST, GHOST)), mode="wrap")


def run_periodic(U, dx, nsteps, cfg=None, dts=None):
    """nsteps steps with each step's dt from the CFL condition of its own state (or from dts)."""
    used = []
    for n in range(nsteps):
        dt = cfl_periodic(U, dx, cfg) if dts is None else dts[n]
        U = step_periodic(U, dx, dt, cfg)
        used.append(dt)
    return U, used
