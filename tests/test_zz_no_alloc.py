"""The allocation-free batched step (hydro_step_batched_noalloc), for callers that cannot allocate
device memory, called through the C ABI.  It runs the kernels and work-list of hydro_step at tile
0 with 32-plane z chunks, so two calls in a row must give the bits of the context-based hydro_step
at that tuning (states and fused dt).  Collected last on purpose: it shares file-scope device
scratch with nothing else, but a failure here should not hide the other tests' results."""
import numpy as np
import pytest
import torch

import workloads

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu


def _batch(dtype):
    parent = workloads.turbulent_state(32, seed=11, mach=3.0, sedov=False)
    descs = workloads.patch_set(12, seed=11, edges=(4, 8, 12, 16, 24, 40), max_level=2)
    origins = workloads.patch_origins(descs, parent.shape[1:], seed=11)
    ins, outs_ref, outs_na = [], [], []
    for d, o in zip(descs, origins):
        Ug = workloads.ghosted_from_periodic(parent, o, (d["nx"], d["ny"], d["nz"])).to("cuda", dtype).contiguous()
        ins.append(hy.patch(Ug, 2, d["dx"], d["level"]))
        outs_ref.append(hy.patch(torch.zeros_like(Ug), 2, d["dx"], d["level"]))
        outs_na.append(hy.patch(torch.zeros_like(Ug), 2, d["dx"], d["level"]))
    return ins, outs_ref, outs_na


def _cfg(precision):
    cfg = hy.hydro_config()
    cfg.gamma, cfg.cfl, cfg.rho_floor, cfg.p_floor = 5.0 / 3.0, 0.8, 1e-10, 1e-14
    cfg.limiter = hy.HYDRO_MINMOD
    cfg.precision = hy.PRECISIONS[precision]
    cfg.cuda_stream = torch.cuda.current_stream().cuda_stream
    return cfg


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
def test_noalloc_step_matches_context_step_twice(precision):
    dtype = torch.float32 if precision == "fp32" else torch.float64
    ins, outs_ref, outs_na = _batch(dtype)
    n = len(ins)
    c = hy.hydro_init(precision=precision)
    hy.hydro_set_tuning(c, 0, 32)  # the tuning the allocation-free call runs
    dt = torch.empty(n, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, ins, dt)
    dt *= 0.7
    dn_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    hy.hydro_step(c, ins, outs_ref, dt, dn_ref)
    rc, bits = hy.hydro_get_error(c)
    assert rc == hy.HYDRO_OK, bits
    cfg = _cfg(precision)
    a = (hy.hydro_patch * n)(*[p.c for p in ins])
    b = (hy.hydro_patch * n)(*[p.c for p in outs_na])
    for call in range(2):
        for p in outs_na:
            for t in p.tensors:
                t.zero_()
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        dn = torch.empty(n, dtype=torch.float64, device="cuda")
        rc = hy.hydro_step_batched_noalloc(cfg, a, b, n, dt, dn, err)
        assert rc == hy.HYDRO_OK, hy.status_string(rc)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        for pr, pn in zip(outs_ref, outs_na):
            for tr, tn in zip(pr.tensors, pn.tensors):
                assert torch.equal(tr, tn), call
        assert torch.equal(dn, dn_ref), call
    hy.hydro_finalize(c)


def test_noalloc_periodic_box_matches_context_step():
    """A single periodic box (no ghost layers), as hydro_step accepts it."""
    U = workloads.turbulent_state((20, 36, 40), seed=12, mach=3.0, sedov=True).to("cuda").contiguous()
    dx = 1.0 / 40
    c = hy.hydro_init(precision="fp64")
    hy.hydro_set_tuning(c, 0, 32)
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_cfl_dt(c, hy.patch(U, 0, dx), dt)
    ref = torch.empty_like(U)
    dn_ref = torch.empty(1, dtype=torch.float64, device="cuda")
    hy.hydro_step(c, hy.patch(U, 0, dx), hy.patch(ref, 0, dx), dt, dn_ref)
    torch.cuda.synchronize()
    got = torch.empty_like(U)
    a = (hy.hydro_patch * 1)(hy.patch(U, 0, dx).c)
    b = (hy.hydro_patch * 1)(hy.patch(got, 0, dx).c)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    dn = torch.empty(1, dtype=torch.float64, device="cuda")
    assert hy.hydro_step_batched_noalloc(_cfg("fp64"), a, b, 1, dt, dn, err) == hy.HYDRO_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(got, ref) and torch.equal(dn, dn_ref)
    hy.hydro_finalize(c)


def test_noalloc_reports_device_errors_in_the_callers_word():
    ins, _, outs = _batch(torch.float64)
    n = len(ins)
    cfg = _cfg("fp64")
    a = (hy.hydro_patch * n)(*[p.c for p in ins])
    b = (hy.hydro_patch * n)(*[p.c for p in outs])
    dt = torch.zeros(n, dtype=torch.float64, device="cuda")  # dt = 0: flagged on the device
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert hy.hydro_step_batched_noalloc(cfg, a, b, n, dt, None, err) == hy.HYDRO_OK
    torch.cuda.synchronize()
    assert int(err.item()) & hy.EBIT_BAD_DT
    # no error word: refused before any launch
    assert hy.hydro_step_batched_noalloc(cfg, a, b, n, dt, None, None) == hy.HYDRO_ERR_ARG


def test_noalloc_rejects_oversized_batches():
    ins, _, outs = _batch(torch.float64)
    cfg = _cfg("fp64")
    big = 5000  # above the 4096-patch maximum of the static scratch
    a = (hy.hydro_patch * big)(*([ins[0].c] * big))
    b = (hy.hydro_patch * big)(*([outs[0].c] * big))
    dt = torch.ones(big, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert hy.hydro_step_batched_noalloc(cfg, a, b, big, dt, None, err) == hy.HYDRO_ERR_ARG
    np.testing.assert_array_equal(err.cpu().numpy(), [0])
