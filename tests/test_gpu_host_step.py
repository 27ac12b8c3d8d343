"""hydro_step_host (a periodic box in host memory; copies pipelined with the step over z slabs)
against hydro_step on the same state held on the device: bitwise equal states and fused CFL dt
over two chained calls (ping-pong host buffers), for ragged slab counts and every precision;
page-locked and pageable host memory; argument errors."""
import ctypes

import pytest
import torch

import workloads
from hydro_testlib import check_clean, ctx

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu


def _device_steps(c, U, dx, nsteps):
    a = U.cuda()
    d = torch.empty(nsteps + 1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(a, 0, dx), d[0:1])
    outs = []
    for n in range(nsteps):
        b = torch.empty_like(a)
        hy.hydro_step(c, hy.patch(a, 0, dx), hy.patch(b, 0, dx), d[n:n + 1], d[n + 1:n + 2])
        outs.append(b)
        a = b
    torch.cuda.synchronize()
    return [o.cpu() for o in outs], d.cpu()


def _host_steps(c, U, dx, nsteps, dt0, pinned=True):
    bufs = [U.clone(), torch.empty_like(U), torch.empty_like(U)]
    if pinned:
        bufs = [t.pin_memory() for t in bufs]
    d = torch.empty(nsteps + 1, dtype=torch.float64, device="cuda")
    d[0] = dt0
    outs = []
    for n in range(nsteps):
        src, dst = bufs[n % 3], bufs[(n + 1) % 3]
        hy.hydro_step_host(c, hy.host_patch(src, dx), hy.host_patch(dst, dx), d[n:n + 1], d[n + 1:n + 2])
        outs.append(dst)
    torch.cuda.synchronize()
    return [o.clone() for o in outs], d.cpu()


@pytest.mark.parametrize("precision", ["fp64", "df64", "fp32", "mixed"])
@pytest.mark.parametrize("shape", [(70, 17, 33), (37, 20, 18), (3, 9, 10), (1, 6, 7)])
def test_host_step_equals_device_step(precision, shape):
    c = ctx(precision)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    U = workloads.turbulent_state(shape, seed=2, mach=5.0, sedov=True).to(dtype).contiguous()
    dx = 1.0 / shape[2]
    want, wd = _device_steps(c, U, dx, 2)
    got, gd = _host_steps(c, U, dx, 2, wd[0].item())
    for g, w in zip(got, want):
        assert torch.equal(g, w)
    assert torch.equal(gd, wd)


@pytest.mark.parametrize("zchunk", [1, 2, 3, 8])
def test_host_step_small_slabs(zchunk):
    """Slabs of one to eight planes (one-plane chunks are widened to two, so that a slab's upper
    halo lies in the next slab), each slab's step started by the arrival of the next slab's first
    two planes, consecutive slabs on alternating compute streams: the same bits as hydro_step."""
    c = ctx("fp64")
    shape = (29, 12, 14)
    U = workloads.turbulent_state(shape, seed=3, mach=5.0, sedov=True).contiguous()
    dx = 1.0 / 14
    want, wd = _device_steps(c, U, dx, 2)
    hy.hydro_set_tuning(c, 0, zchunk)
    got, gd = _host_steps(c, U, dx, 2, wd[0].item())
    for g, w in zip(got, want):
        assert torch.equal(g, w)
    assert torch.equal(gd, wd)
    check_clean(c)


@pytest.mark.parametrize("zchunk,nz", [(8, 128), (8, 130), (8, 133), (16, 262)])
@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_host_step_ramped_slabs(precision, zchunk, nz):
    """Boxes tall enough for slabs of the tuned z chunk ramped at both ends (zc/4, zc/2, ..., zc/2,
    zc/4 planes; a left-over of one plane merged into the last full slab, of more into a slab of its
    own): the same bits as hydro_step."""
    c = ctx(precision)
    shape = (nz, 12, 14)
    U = workloads.turbulent_state(shape, seed=4, mach=5.0, sedov=True).contiguous()
    dx = 1.0 / 14
    want, wd = _device_steps(c, U, dx, 2)
    hy.hydro_set_tuning(c, 0, zchunk)
    got, gd = _host_steps(c, U, dx, 2, wd[0].item())
    for g, w in zip(got, want):
        assert torch.equal(g, w)
    assert torch.equal(gd, wd)
    check_clean(c)


def test_host_step_pageable_memory():
    c = ctx("fp64")
    U = workloads.turbulent_state((24, 16, 16), seed=3, mach=2.0, sedov=False).contiguous()
    dx = 1.0 / 16
    want, wd = _device_steps(c, U, dx, 2)
    got, gd = _host_steps(c, U, dx, 2, wd[0].item(), pinned=False)
    for g, w in zip(got, want):
        assert torch.equal(g, w)
    assert torch.equal(gd, wd)
    check_clean(c)


def test_host_step_rejects_device_pointers_and_ghosts():
    c = ctx("fp64")
    a = torch.zeros((5, 8, 8, 8), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    d = torch.ones(2, dtype=torch.float64, device="cuda")
    pa, pb = hy.patch(a, 0, 0.125), hy.patch(b, 0, 0.125)
    rc = hy.lib().hydro_step_host(c.handle, ctypes.byref(pa.c), ctypes.byref(pb.c), d.data_ptr(), None)
    assert rc == hy.HYDRO_ERR_ARG
    h = torch.zeros((5, 12, 12, 12), dtype=torch.float64).pin_memory()
    g = torch.zeros_like(h).pin_memory()
    ph, pg = hy.Patch(h, 2, 0.125, host=True), hy.Patch(g, 2, 0.125, host=True)
    rc = hy.lib().hydro_step_host(c.handle, ctypes.byref(ph.c), ctypes.byref(pg.c), d.data_ptr(), None)
    assert rc == hy.HYDRO_ERR_ARG
    with pytest.raises(ValueError):
        hy.host_patch(a, 0.125)
