"""The bounds-checked build (libhydro_checked.so, compiled with HYDRO_CHECK_BOUNDS): every global index of
the step kernels and of the fused MHD tile kernel is tested against its array's extent and an index
outside sets HYDRO_EBIT_OOB (the access skipped).  A sanitizer stand-in that faults nothing: the same
steps -- periodic boxes of odd sizes, ghosted patches of odd sizes stored as unaligned views with odd
strides, every tile shape, several z chunks, a tile shape per patch class, MHD boxes and patches, four
precisions -- run through the checked library (in a child process that loads it) and through the
default one; the checked run raises no bit and gives the same bits."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_cases(hy):
    """Every case's outputs (and the OR of the error bits) as numpy arrays."""
    import workloads
    out, bits = {}, 0
    for precision in ("fp64", "df64", "fp32", "mixed"):
        dtype = torch.float32 if precision == "fp32" else torch.float64
        c = hy.hydro_init(precision=precision)
        for si, shape in enumerate([(12, 40, 70), (37, 21, 19), (5, 3, 37)]):
            U = workloads.turbulent_state(shape, seed=si, mach=3.0, sedov=True).to("cuda", dtype).contiguous()
            dt = torch.empty(1, dtype=torch.float64, device="cuda")
            hy.hydro_cfl_dt(c, hy.patch(U, 0, 1.0 / shape[2]), dt)
            for tile in range(hy.NUM_TILES):
                for zc in (8, 5):
                    hy.hydro_set_tuning(c, tile, zc)
                    V = torch.empty_like(U)
                    hy.hydro_step(c, hy.patch(U, 0, 1.0 / shape[2]), hy.patch(V, 0, 1.0 / shape[2]), dt)
                    out["%s_box%d_t%d_z%d" % (precision, si, tile, zc)] = V.double().cpu().numpy()
        # ghosted patches of odd sizes as views with odd strides, one element into their buffers
        parent = workloads.turbulent_state(16, seed=8, mach=3.0, sedov=False)
        dims = [(5, 7, 9), (13, 3, 11), (1, 1, 1), (17, 19, 6), (8, 24, 16), (32, 16, 9)]
        origins = [(3, 5, 7), (15, 0, 2), (8, 8, 8), (0, 11, 13), (4, 4, 4), (9, 1, 6)]
        ins, outs = [], []
        for (nx, ny, nz), o in zip(dims, origins):
            Ug = workloads.ghosted_from_periodic(parent, o, (nx, ny, nz)).to("cuda", dtype)
            F, Z, Y, X = Ug.shape
            bi = torch.zeros((F, Z, Y, X + 2), dtype=dtype, device="cuda")
            bo = torch.zeros((F, Z, Y, X + 4), dtype=dtype, device="cuda")
            bi[:, :, :, 1:1 + X].copy_(Ug)
            ins.append(hy.patch(bi[:, :, :, 1:1 + X], 2, 1.0 / 64))
            outs.append(hy.patch(bo[:, :, :, 1:1 + X], 2, 1.0 / 64))
        dtp = torch.empty(len(ins), dtype=torch.float64, device="cuda")
        hy.hydro_cfl_dt(c, ins, dtp)
        for tile in range(hy.NUM_TILES):
            hy.hydro_set_tuning(c, tile, 4)
            hy.hydro_step(c, ins, outs, dtp)
            for k, po in enumerate(outs):
                out["%s_patch%d_t%d" % (precision, k, tile)] = torch.stack(po.tensors).double().cpu().numpy()
        for k, (t, z) in enumerate([(2, 3), (1, 5), (3, 16)]):
            hy.hydro_set_class_tuning(c, k, t, z)
        hy.hydro_step(c, ins, outs, dtp)
        for k, po in enumerate(outs):
            out["%s_patch%d_classes" % (precision, k)] = torch.stack(po.tensors).double().cpu().numpy()
        # MHD (one fused tile kernel in float arithmetic): periodic boxes of odd sizes, then ghosted
        # patches of odd sizes stored as views with odd strides, one element into their buffers
        for si, shape in enumerate([(13, 21, 35), (5, 9, 3)]):
            Um = workloads.mhd_state(shape, seed=70 + si, beta=0.5, mach=1.5, psi_amp=0.05)
            Um = Um.to("cuda", dtype).contiguous()
            dx = 1.0 / shape[2]
            dm = torch.empty(2, dtype=torch.float64, device="cuda")
            hy.hydro_mhd_cfl_dt(c, Um, dx, dm[0:1])
            Vm = torch.empty_like(Um)
            hy.hydro_mhd_step(c, Um, Vm, dx, dm[0:1], dm[1:2])
            out["%s_mhd_box%d" % (precision, si)] = Vm.double().cpu().numpy()
            out["%s_mhd_box%d_dt" % (precision, si)] = dm.cpu().numpy()
        mparent = workloads.mhd_state((18, 14, 22), seed=72, beta=0.5, mach=1.5, psi_amp=0.05)
        mins, mouts = [], []
        for k, ((nx, ny, nz), o) in enumerate(zip([(35, 9, 5), (3, 17, 11), (1, 1, 2)],
                                                   [(2, 3, 4), (10, 0, 7), (5, 5, 5)])):
            Ug = workloads.ghosted_from_periodic(mparent, o, (nx, ny, nz)).to("cuda", dtype)
            F, Z, Y, X = Ug.shape
            gout = 2 * (k % 2)
            bi = torch.zeros((F, Z, Y, X + 2), dtype=dtype, device="cuda")
            bo = torch.zeros((F, nz + 2 * gout, ny + 2 * gout, nx + 2 * gout + 3), dtype=dtype, device="cuda")
            bi[:, :, :, 1:1 + X].copy_(Ug)
            mins.append(hy.MhdPatch(bi[:, :, :, 1:1 + X], 2, 1.0 / 32))
            mouts.append(hy.MhdPatch(bo[:, :, :, 1:1 + nx + 2 * gout], gout, 1.0 / 32))
        dtm = torch.empty(2 * len(mins), dtype=torch.float64, device="cuda")
        hy.hydro_mhd_cfl_patches(c, mins, dtm[:len(mins)])
        hy.hydro_mhd_step_patches(c, mins, mouts, dtm[:len(mins)], dtm[len(mins):])
        for k, po in enumerate(mouts):
            out["%s_mhd_patch%d" % (precision, k)] = torch.stack(po.tensors).double().cpu().numpy()
        out["%s_mhd_patch_dt" % precision] = dtm.cpu().numpy()
        rc, b = hy.hydro_get_error(c)
        bits |= b
        hy.hydro_finalize(c)
    out["bits"] = np.array([bits])
    return out


CHILD = """
import sys, numpy as np
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import paper_1412_0934_gb300 as hy
import test_gpu_checked_build as m
assert hy.LIB_PATH.endswith("libhydro_checked.so"), hy.LIB_PATH
np.savez({path!r}, **m.run_cases(hy))
"""


def test_checked_build_flags_nothing_and_matches_the_default_build(tmp_path):
    from paper_1412_0934_gb300 import build
    lib, _ = build.build(checked=True)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, HYDRO_LIBRARY=lib)
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=path)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    import paper_1412_0934_gb300 as hy
    assert not hy.LIB_PATH.endswith("libhydro_checked.so")
    ref = run_cases(hy)
    got = np.load(path)
    assert int(got["bits"][0]) == 0 and int(ref["bits"][0]) == 0, (int(got["bits"][0]), int(ref["bits"][0]))
    assert set(got.files) == set(ref)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
