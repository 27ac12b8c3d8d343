"""GPU flux registers, refluxing and average-down against the oracle (oracle.patch_boundary_fluxes,
oracle/amr.py): registers of ghosted patches per precision; registers of level boxes equal to the
same boxes cut out as patches (bitwise); refluxing bitwise and average-down to rounding on random
inputs; and a two-level composite step on the GPU that conserves to round-off and matches the
oracle's composite step."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from hydro_testlib import check_clean, ctx
from oracle import amr

import paper_1412_0934_gb300 as hy

pytestmark = pytest.mark.gpu


def _regs(boxes, dtype, mult=1):
    return [torch.zeros(5 * hy.register_size(*(mult * np.asarray(n))), dtype=dtype, device="cuda") for n in boxes]


@pytest.mark.parametrize("precision", ["fp64", "df64", "mixed", "fp32"])
def test_patch_registers_match_oracle(precision):
    dtype = torch.float32 if precision == "fp32" else torch.float64
    c = ctx(precision)
    level = workloads.turbulent_state((12, 14, 16), seed=41, mach=3.0, sedov=False)
    dx = 1.0 / 16
    dt = 0.5 * oracle.cfl_periodic(level.numpy(), dx, oracle.config())
    rng = np.random.default_rng(42)
    dims = [(int(rng.integers(1, 9)), int(rng.integers(1, 9)), int(rng.integers(1, 9))) for _ in range(12)]
    origins = [(int(rng.integers(0, 16)), int(rng.integers(0, 14)), int(rng.integers(0, 12))) for _ in dims]
    pats = [workloads.ghosted_from_periodic(level, o, n).to(dtype).contiguous() for o, n in zip(origins, dims)]
    regs = _regs(dims, dtype)
    dts = torch.full((len(dims),), dt, dtype=torch.float64, device="cuda")
    hy.hydro_patch_fluxes(c, [hy.patch(p.cuda(), 2, dx) for p in pats], dts, regs)
    torch.cuda.synchronize()
    tol = {"fp64": 1e-12, "df64": 1e-12}.get(precision, 1e-5)
    for p, r in zip(pats, regs):
        want = dt * oracle.patch_boundary_fluxes(p.double().numpy(), dx, dt)
        got = r.double().cpu().numpy().reshape(5, -1)
        err = np.abs(got - want).max(axis=1) / np.maximum(np.abs(want).max(axis=1), 1e-300)
        assert err.max() <= tol, err
    check_clean(c)


def test_level_box_registers_equal_patch_registers_and_accumulate():
    c = ctx("fp64")
    level = workloads.turbulent_state((10, 12, 14), seed=43, mach=2.0, sedov=False)
    dx = 1.0 / 14
    dt = 0.5 * oracle.cfl_periodic(level.numpy(), dx, oracle.config())
    boxes = [((0, 0, 0), (3, 4, 5)), ((12, 10, 8), (4, 3, 2)), ((5, 6, 7), (1, 1, 1))]  # incl. wrap
    pr = _regs([n for _, n in boxes], torch.float64)
    lr = _regs([n for _, n in boxes], torch.float64)
    dts = torch.full((len(boxes),), dt, dtype=torch.float64, device="cuda")
    pats = [workloads.ghosted_from_periodic(level, o, n).contiguous().cuda() for o, n in boxes]
    hy.hydro_patch_fluxes(c, [hy.patch(p, 2, dx) for p in pats], dts, pr)
    hy.hydro_level_fluxes(c, hy.patch(level.cuda(), 0, dx), [o for o, _ in boxes], [n for _, n in boxes], dts[:1], lr)
    hy.hydro_level_fluxes(c, hy.patch(level.cuda(), 0, dx), [o for o, _ in boxes], [n for _, n in boxes], dts[:1], lr,
                          accumulate=True)
    torch.cuda.synchronize()
    for a, b in zip(pr, lr):
        assert torch.equal(2 * a, b)
    check_clean(c)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_reflux_bitwise_and_average_down_match_oracle(precision):
    dtype = torch.float32 if precision == "fp32" else torch.float64
    c = ctx(precision)
    rng = np.random.default_rng(44)
    Uc = rng.standard_normal((5, 10, 9, 12)) + 3.0
    dxc = 1.0 / 12
    boxes = [((2, 1, 3), (3, 4, 2)), ((8, 5, 0), (4, 2, 3)), ((0, 6, 6), (2, 3, 4))]  # last one wraps in x
    Rc = [rng.standard_normal((5, hy.register_size(*n))) * 1e-3 for _, n in boxes]
    Rf = [rng.standard_normal((5, hy.register_size(*(2 * np.asarray(n))))) * 1e-3 for _, n in boxes]
    Ucd = torch.tensor(Uc, dtype=dtype, device="cuda").contiguous()
    hy.hydro_reflux(c, hy.patch(Ucd, 0, dxc), [o for o, _ in boxes], [n for _, n in boxes],
                    [torch.tensor(r, dtype=dtype, device="cuda").contiguous() for r in Rc],
                    [torch.tensor(r, dtype=dtype, device="cuda").contiguous() for r in Rf])
    torch.cuda.synchronize()
    want = np.array(Uc, dtype=np.float32 if precision == "fp32" else np.float64).astype(np.float64)
    for (o, n), rc, rf in zip(boxes, Rc, Rf):
        cast = (lambda a: a.astype(np.float32).astype(np.float64)) if precision == "fp32" else (lambda a: a)
        want = amr.reflux(want, o, n, cast(rc), cast(rf), dxc)
    got = Ucd.double().cpu().numpy()
    if precision == "fp64":
        assert np.array_equal(got, want)
    else:
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
    # average-down of fine patches (origins and sizes even)
    fines = [((4, 2, 6), (6, 8, 4)), ((16, 10, 0), (8, 4, 6))]
    Fi = [rng.standard_normal((5, n[2], n[1], n[0])) + 2.0 for _, n in fines]
    tens = []
    for (o, n), f in zip(fines, Fi):
        t = torch.zeros((5, n[2] + 4, n[1] + 4, n[0] + 4), dtype=dtype)
        t[:, 2:-2, 2:-2, 2:-2] = torch.tensor(f, dtype=dtype)
        tens.append(t.cuda())
    hy.hydro_average_down(c, hy.patch(Ucd, 0, dxc), [hy.patch(t, 2, dxc / 2) for t in tens], [o for o, _ in fines])
    torch.cuda.synchronize()
    for (o, n), t in zip(fines, tens):
        want = amr.average_down(want, t[:, 2:-2, 2:-2, 2:-2].double().cpu().numpy(), tuple(v // 2 for v in o))
    got = Ucd.double().cpu().numpy()
    assert np.abs(got - want).max() <= (1e-15 if precision == "fp64" else 1e-6) * np.abs(want).max()


def test_two_level_composite_step_conserves_on_the_gpu():
    """Coarse 16^3 periodic level, a fine patch over the coarse box [4, 12)^3: coarse step with its
    box register, two fine substeps (ghosts prolonged at t and, linearly in time, at t + dt/2)
    accumulating the fine register, refluxing, average-down.  The composite totals are conserved
    to round-off and the coarse level matches the oracle's composite step."""
    import test_oracle_amr as ref
    U0, want = ref._composite_step(True)
    c = ctx("fp64")
    dxc = 1.0 / 16
    cfg = oracle.config()
    dtc = 0.5 * oracle.cfl_periodic(U0, dxc, cfg)
    Uc = torch.tensor(U0, device="cuda").contiguous()
    Uc1 = torch.empty_like(Uc)
    d = torch.tensor([dtc, dtc / 2], dtype=torch.float64, device="cuda")
    oc, nc = (4, 4, 4), (8, 8, 8)
    Rc = _regs([nc], torch.float64)
    Rf = _regs([nc], torch.float64, mult=2)
    hy.hydro_level_fluxes(c, hy.patch(Uc, 0, dxc), [oc], [nc], d[:1], Rc)
    hy.hydro_step(c, hy.patch(Uc, 0, dxc), hy.patch(Uc1, 0, dxc), d[:1])
    Uf = torch.tensor(amr.prolong_box(U0)[:, 8:24, 8:24, 8:24], device="cuda")
    for sub, Ut in enumerate((Uc, 0.5 * (Uc + Uc1))):
        Ug = torch.zeros((5, 20, 20, 20), dtype=torch.float64, device="cuda")
        Ug[:, 2:-2, 2:-2, 2:-2] = Uf
        Vg = torch.zeros_like(Ug)
        pg = hy.patch(Ug, 2, dxc / 2)
        hy.hydro_fill_ghosts(c, hy.patch(Ut.contiguous(), 0, dxc), [pg], [(8, 8, 8)])
        hy.hydro_patch_fluxes(c, [pg], d[1:], Rf, accumulate=sub > 0)
        hy.hydro_step(c, [pg], [hy.patch(Vg, 2, dxc / 2)], d[1:])
        Uf = Vg[:, 2:-2, 2:-2, 2:-2].clone()
    fine = torch.zeros((5, 20, 20, 20), dtype=torch.float64, device="cuda")
    fine[:, 2:-2, 2:-2, 2:-2] = Uf
    hy.hydro_reflux(c, hy.patch(Uc1, 0, dxc), [oc], [nc], Rc, Rf)
    hy.hydro_average_down(c, hy.patch(Uc1, 0, dxc), [hy.patch(fine, 2, dxc / 2)], [(8, 8, 8)])
    torch.cuda.synchronize()
    got = Uc1.cpu().numpy()
    scale = np.abs(U0).sum(axis=(1, 2, 3))
    drift = np.abs(got.sum(axis=(1, 2, 3)) - U0.sum(axis=(1, 2, 3))) / scale
    assert drift.max() <= 1e-14, drift
    err = np.abs(got - want).max(axis=(1, 2, 3)) / np.abs(want).max(axis=(1, 2, 3))
    assert err.max() <= 1e-12, err
    check_clean(c)
