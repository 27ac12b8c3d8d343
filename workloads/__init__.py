"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module holds no arithmetic of the hydro scheme: it draws random fields and builds
conserved states from primitive ones (rho, rho*v, p/(gamma-1) + rho|v|^2/2, the definition of
the conserved variables of an ideal gas).  The oracle and the CUDA library each take these
arrays as inputs; neither imports the other.

The shapes and value distributions stand in for the paper's cosmological runs (its data are
not available): lognormal densities, Gaussian random velocities with a k^-4 power spectrum at
a given rms Mach number, cold gas (small P/rho), a point blast, AMR patch sets with mixed
shapes and levels, and Ramses-style oct groups with a gathered 6^3 stencil.

All generators work with torch on CPU or CUDA (``device``) and are seeded; arrays are float64
of shape (5, nz, ny, nx), fields (rho, m_x, m_y, m_z, E), x fastest.
"""
import math

import numpy as np
import torch

GAMMA = 5.0 / 3.0


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def cons_from_prim(rho, vx, vy, vz, p, gamma=GAMMA):
    """Conserved state (5, ...) from primitive fields (tensors of one shape)."""
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return torch.stack([rho, rho * vx, rho * vy, rho * vz, E])


def lognormal_density(shape, sigma, gen, device):
    """rho = exp(sigma g - sigma^2/2), g ~ N(0,1) per cell (mean 1)."""
    g = torch.randn(shape, generator=gen, device=device, dtype=torch.float64)
    return torch.exp(sigma * g - 0.5 * sigma * sigma)


def powerlaw_velocity(shape, slope_power, gen, device):
    """Three independent Gaussian random fields with power spectrum |v(k)|^2 ~ k^slope_power,
    k = 0 removed, each normalised to unit variance before the caller scales them."""
    nz, ny, nx = shape
    kz = torch.fft.fftfreq(nz, device=device, dtype=torch.float64) * nz
    ky = torch.fft.fftfreq(ny, device=device, dtype=torch.float64) * ny
    kx = torch.fft.rfftfreq(nx, device=device, dtype=torch.float64) * nx
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (slope_power / 4.0), torch.zeros_like(k2))
    out = []
    for _ in range(3):
        w = torch.randn(shape, generator=gen, device=device, dtype=torch.float64)
        f = torch.fft.rfftn(w) * amp
        v = torch.fft.irfftn(f, s=shape)
        v = v - v.mean()
        v = v / v.pow(2).mean().sqrt()
        out.append(v)
        del w, f
    return out


def white_velocity_state(n=32, seed=1, sigma_rho=0.5, p0=1.0, vel_frac=0.3, gamma=GAMMA, p_jitter=0.0,
                         device="cpu"):
    """Lognormal density (mean 1), white Gaussian velocities with sigma = vel_frac * c_s,
    c_s = sqrt(gamma p0 / <rho>), mean removed, uniform pressure p0 (the 32^3 FP64 case), or with
    p_jitter > 0 a pressure p0 * exp(p_jitter g - p_jitter^2/2) per cell."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    gen = _gen(seed, device)
    rho = lognormal_density(shape, sigma_rho, gen, device)
    cs = math.sqrt(gamma * p0 / 1.0)
    v = []
    for _ in range(3):
        c = torch.randn(shape, generator=gen, device=device, dtype=torch.float64) * (vel_frac * cs)
        v.append(c - c.mean())
    p = torch.full(shape, p0, dtype=torch.float64, device=device)
    if p_jitter > 0:
        p = p * lognormal_density(shape, p_jitter, gen, device)
    return cons_from_prim(rho, v[0], v[1], v[2], p, gamma)


def turbulent_state(n, seed=2, mach=5.0, sigma_rho=1.0, p_over_rho=1e-4, sedov=True, gamma=GAMMA,
                    device="cpu"):
    """Cold turbulent gas: k^-4 velocities at 3D rms Mach number `mach` (c_s = sqrt(gamma P/rho),
    uniform since P/rho is), lognormal density, P = p_over_rho * rho, and optionally a Sedov
    point blast adding E = 1 (energy density 1/dx^3, dx = 1/n) to cell (n/2, n/2, n/2)."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    gen = _gen(seed, device)
    rho = lognormal_density(shape, sigma_rho, gen, device)
    cs = math.sqrt(gamma * p_over_rho)
    vx, vy, vz = powerlaw_velocity(shape, -4.0, gen, device)
    scale = mach * cs / math.sqrt(3.0)  # each unit-variance component -> 3D rms = mach * cs
    U = cons_from_prim(rho, vx * scale, vy * scale, vz * scale, p_over_rho * rho, gamma)
    del vx, vy, vz
    if sedov:
        nz, ny, nx = shape
        dx = 1.0 / nx
        U[4, nz // 2, ny // 2, nx // 2] += 1.0 / dx ** 3
    return U


def sound_wave(shape, amp=1e-3, kvec=(1, 1, 0), rho0=1.0, c0=1.0, gamma=GAMMA, phase=0.0, device="cpu"):
    """Right-moving linear sound wave on the unit box (periodic): delta rho = amp rho0 sin(2 pi k.x + phase),
    v = c0 amp sin(.) k_hat, delta p = c0^2 delta rho, around p0 = rho0 c0^2/gamma.
    A phase that is not a multiple of pi/4 avoids cells with exactly equal values around the
    extrema (which put limited slopes exactly on their kink).  Returns (U, period)."""
    nz, ny, nx = shape
    x = (torch.arange(nx, device=device, dtype=torch.float64) + 0.5) / nx
    y = (torch.arange(ny, device=device, dtype=torch.float64) + 0.5) / ny
    z = (torch.arange(nz, device=device, dtype=torch.float64) + 0.5) / nz
    kx, ky, kz = kvec
    ph = 2 * math.pi * (kx * x[None, None, :] + ky * y[None, :, None] + kz * z[:, None, None]) + phase
    s = torch.sin(ph)
    kn = math.sqrt(kx * kx + ky * ky + kz * kz)
    p0 = rho0 * c0 * c0 / gamma
    rho = rho0 * (1 + amp * s)
    vmag = c0 * amp * s
    U = cons_from_prim(rho, vmag * kx / kn, vmag * ky / kn, vmag * kz / kn, p0 + c0 * c0 * rho0 * amp * s, gamma)
    return U, 1.0 / (kn * c0)


def riemann_1d(n, left, right, axis=0, ntrans=4, gamma=GAMMA, device="cpu"):
    """Shock tube along `axis` (0=x,1=y,2=z) on n cells, interface at 0.5, ntrans cells in the
    other two directions.  left/right are (rho, u, p) with u along the axis."""
    shape = [ntrans, ntrans, ntrans]
    shape[2 - axis] = n  # array order is (z, y, x)
    xc = (torch.arange(n, device=device, dtype=torch.float64) + 0.5) / n
    is_left = (xc < 0.5).to(torch.float64)
    view = [1, 1, 1]
    view[2 - axis] = n
    L = is_left.view(view).expand(shape)
    rho = left[0] * L + right[0] * (1 - L)
    un = left[1] * L + right[1] * (1 - L)
    p = left[2] * L + right[2] * (1 - L)
    v = [torch.zeros(shape, dtype=torch.float64, device=device) for _ in range(3)]
    v[axis] = un
    return cons_from_prim(rho, v[0], v[1], v[2], p, gamma)


def sedov_blast(n, rho0=1.0, p_amb=1e-5, E=1.0, gamma=GAMMA, device="cpu"):
    """Uniform cold gas with energy E deposited in cell (n/2, n/2, n/2) of the unit box."""
    shape = (n, n, n)
    rho = torch.full(shape, rho0, dtype=torch.float64, device=device)
    z = torch.zeros(shape, dtype=torch.float64, device=device)
    U = cons_from_prim(rho, z, z, z, torch.full(shape, p_amb, dtype=torch.float64, device=device), gamma)
    U[4, n // 2, n // 2, n // 2] += E * n ** 3
    return U


def ghosted_from_periodic(U, origin, dims, ghost=2):
    """Ghosted box of interior `dims` (nx, ny, nz) at `origin` (x, y, z) cut from the periodic field U,
    ghosts filled from the field itself (exact ghosts).  Returns (5, nz+2g, ny+2g, nx+2g)."""
    _, NZ, NY, NX = U.shape
    ox, oy, oz = origin
    nx, ny, nz = dims
    dev = U.device
    ix = (torch.arange(ox - ghost, ox + nx + ghost, device=dev) % NX)
    iy = (torch.arange(oy - ghost, oy + ny + ghost, device=dev) % NY)
    iz = (torch.arange(oz - ghost, oz + nz + ghost, device=dev) % NZ)
    return U[:, iz][:, :, iy][:, :, :, ix]


PATCH_EDGES = (8, 16, 24, 32, 48)


def patch_set(npatch=4096, seed=3, edges=PATCH_EDGES, max_level=5, base_dx=1.0 / 64.0):
    """AMR patch descriptors: half cubes n^3, half 2:1 boxes with the long axis (2n) uniform over
    x, y, z; n uniform over `edges`; level uniform over 0..max_level, dx = base_dx * 2^-level.
    Returns a list of dicts (nx, ny, nz, level, dx)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(npatch):
        n = int(rng.choice(edges))
        dims = [n, n, n]
        if i % 2 == 1:
            dims[int(rng.integers(0, 3))] = 2 * n
        level = int(rng.integers(0, max_level + 1))
        out.append(dict(nx=dims[0], ny=dims[1], nz=dims[2], level=level, dx=base_dx * 2.0 ** (-level)))
    return out


def patch_origins(patches, parent_shape, seed=3):
    """Random origins (x, y, z) inside the periodic parent for each patch."""
    rng = np.random.default_rng(seed + 1000)
    NZ, NY, NX = parent_shape
    return [(int(rng.integers(0, NX)), int(rng.integers(0, NY)), int(rng.integers(0, NZ))) for _ in patches]


def oct_origins(ngroups, parent_shape, seed=3):
    """Origins (x, y, z) of 2^3 octs on even coordinates of the periodic parent."""
    rng = np.random.default_rng(seed + 2000)
    NZ, NY, NX = parent_shape
    ox = rng.integers(0, NX // 2, ngroups) * 2
    oy = rng.integers(0, NY // 2, ngroups) * 2
    oz = rng.integers(0, NZ // 2, ngroups) * 2
    return np.stack([ox, oy, oz], axis=1)


def gather_octs(U, origins, ghost=2):
    """Gathered 6^3 stencils of the 2^3 octs at `origins` (G, 3) from the periodic field U:
    returns (5, G, 6, 6, 6) -- per field, per group, a ghosted 2^3 box (z, y, x)."""
    _, NZ, NY, NX = U.shape
    dev = U.device
    o = torch.as_tensor(np.asarray(origins), device=dev, dtype=torch.long)
    r = torch.arange(-ghost, 2 + ghost, device=dev)
    ix = (o[:, 0, None] + r[None, :]) % NX  # (G, 6)
    iy = (o[:, 1, None] + r[None, :]) % NY
    iz = (o[:, 2, None] + r[None, :]) % NZ
    flat = (iz[:, :, None, None] * NY + iy[:, None, :, None]) * NX + ix[:, None, None, :]  # (G,6,6,6)
    return U.reshape(5, -1)[:, flat]


def mhd_state(shape, seed=1, beta=1.0, mach=1.0, psi_amp=0.01, modes=6, gamma=GAMMA, device="cpu"):
    """Smooth periodic magnetised gas for the MHD step: each primitive field a sum of `modes` random
    Fourier modes (wavenumbers 0..3 per axis, not all zero) on the unit box.  rho = 1 + 0.1 f (mean 1),
    p = 1 + 0.1 g, velocities of rms Mach `mach` (sound speed of the mean state), B of rms
    sqrt(2 <p> / beta) (plasma beta), psi of amplitude psi_amp; B is not divergence-free.  The mode
    parameters come from a seeded numpy generator; the fields are formed with torch on `device`.
    Returns the conserved state (9, nz, ny, nx) in float64: rho, m, E = p/(gamma-1) + rho |v|^2/2 +
    |B|^2/2, B, psi."""
    if isinstance(shape, int):
        shape = (shape, shape, shape)
    nz, ny, nx = shape
    rng = np.random.default_rng(seed + 5000)
    f64 = dict(device=device, dtype=torch.float64)
    z = ((torch.arange(nz, **f64) + 0.5) / nz)[:, None, None]
    y = ((torch.arange(ny, **f64) + 0.5) / ny)[None, :, None]
    x = ((torch.arange(nx, **f64) + 0.5) / nx)[None, None, :]

    def field():
        f = torch.zeros(shape, **f64)
        for _ in range(modes):
            k = rng.integers(0, 4, 3)
            if not k.any():
                k[rng.integers(0, 3)] = 1
            ph = float(rng.uniform(0, 2 * math.pi))
            a = float(rng.normal())
            f += a * torch.sin(2 * math.pi * (float(k[0]) * x + float(k[1]) * y + float(k[2]) * z) + ph)
        return f / torch.sqrt((f * f).mean()).clamp_min(1e-300)

    rho = 1.0 + 0.1 * field()
    p = 1.0 + 0.1 * field()
    cs = math.sqrt(gamma)
    v = [mach * cs / math.sqrt(3.0) * field() for _ in range(3)]
    b0 = math.sqrt(2.0 / beta) / math.sqrt(3.0)
    B = [b0 * field() for _ in range(3)]
    psi = psi_amp * field()
    E = p / (gamma - 1.0) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2) + 0.5 * (B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
    return torch.stack([rho, rho * v[0], rho * v[1], rho * v[2], E, B[0], B[1], B[2], psi])
