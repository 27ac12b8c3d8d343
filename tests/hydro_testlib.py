"""Helpers shared by the GPU tests: run the library through its C ABI on seeded inputs and
compare with the FP64 oracle."""
import numpy as np
import torch

import paper_1412_0934_gb300 as hy

GAMMA = 5.0 / 3.0


def normwise(g, o):
    """Per-field max|g - o| / max|o| (the parity metric)."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    return np.array([np.abs(g[f] - o[f]).max() / max(np.abs(o[f]).max(), 1e-300) for f in range(5)])


def ctx(precision="fp64", limiter="minmod", **kw):
    return hy.hydro_init(gamma=kw.pop("gamma", GAMMA), limiter=limiter, precision=precision, **kw)


def dev(U, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(U)).to(device="cuda", dtype=dtype).contiguous()


def dts(*vals):
    return torch.tensor(list(vals), dtype=torch.float64, device="cuda")


def step_periodic(c, U, dx, dt, dt_next=False):
    """One uniform periodic step on the GPU; returns (U_next numpy, dt_next or None)."""
    a = dev(U, c.dtype)
    b = torch.empty_like(a)
    d = dts(dt)
    dn = torch.empty(1, dtype=torch.float64, device="cuda") if dt_next else None
    hy.hydro_step(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), d, dn)
    torch.cuda.synchronize()
    return b.double().cpu().numpy(), (dn.item() if dt_next else None)


def cfl(c, U, dx, ng=0):
    a = dev(U, c.dtype)
    d = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(a, ng, dx), d)
    torch.cuda.synchronize()
    return d.item()


def check_clean(c):
    rc, bits = hy.hydro_get_error(c)
    assert rc == hy.HYDRO_OK and bits == 0, "device error bits %#x" % bits
