"""Python binding of libhydro.so, the sm_103a CUDA library declared in include/hydro.h.

Argument marshalling only: every step of the hydro path runs in the library's kernels.  The
functions carry the C ABI's names (hydro_init, hydro_step, hydro_cfl_dt, hydro_step_octs,
hydro_adjoint_step, hydro_run, ...) and take torch CUDA tensors, which own all field memory.
There is no CPU fallback: if the library is not built, or no GPU is present, calls raise.

A patch is built from a tensor of shape (5, nz + 2 ng, ny + 2 ng, nx + 2 ng) (fields rho, m_x,
m_y, m_z, E; x fastest) with ``patch(U, ng, dx)``; float64 for FP64/MIXED, float32 for FP32.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# The library: the in-tree build, or the build the environment variable HYDRO_LIBRARY names (the
# bounds-checked variant libhydro_checked.so, for instance).
LIB_PATH = os.environ.get("HYDRO_LIBRARY") or os.path.join(_HERE, "libhydro.so")

HYDRO_OK = 0
HYDRO_ERR_ARG = -1
HYDRO_ERR_CUDA = -2
HYDRO_ERR_UNPHYSICAL = -3
HYDRO_ERR_TIMEOUT = -4
HYDRO_ERR_NOMEM = -5
HYDRO_ERR_STATE = -6

HYDRO_FP64, HYDRO_FP32, HYDRO_MIXED, HYDRO_FP64_DF = 0, 1, 2, 3
HYDRO_MINMOD, HYDRO_MC, HYDRO_NOLIMIT, HYDRO_PPM = 0, 1, 2, 3
PRECISIONS = {"fp64": HYDRO_FP64, "fp32": HYDRO_FP32, "mixed": HYDRO_MIXED, "df64": HYDRO_FP64_DF}
LIMITERS = {"minmod": HYDRO_MINMOD, "mc": HYDRO_MC, "none": HYDRO_NOLIMIT, "ppm": HYDRO_PPM}

# Compiled tile shapes of the step kernels, by tile id (HYDRO_NUM_TILES in include/hydro.h).
TILE_SHAPES = ((16, 16), (32, 8), (8, 8), (32, 16), (16, 16))
NUM_TILES = len(TILE_SHAPES)
# Patch-shape classes of the per-class tile choice (HYDRO_NUM_PATCH_CLASSES in include/hydro.h).
NUM_PATCH_CLASSES = 3

EBIT_NONFINITE = 0x01
EBIT_RHO_FLOOR = 0x02
EBIT_P_FLOOR = 0x04
EBIT_BAD_DT = 0x08
EBIT_BAD_TILE = 0x10
EBIT_TIMEOUT = 0x20
EBIT_OOB = 0x40

# C symbols that include/hydro.h declares (checked by the tests).
EXPORTS = ("hydro_init", "hydro_finalize", "hydro_cfl_dt", "hydro_step", "hydro_step_host", "hydro_step_octs",
           "hydro_step_octs_level", "hydro_octs_build", "hydro_step_octs_table", "hydro_mhd_step", "hydro_mhd_cfl_dt",
           "hydro_mhd_step_patches", "hydro_mhd_cfl_patches", "hydro_fill_ghosts", "hydro_fill_ghosts_time", "hydro_exchange_ghosts", "hydro_patch_fluxes",
           "hydro_level_fluxes", "hydro_reflux", "hydro_average_down",
           "hydro_adjoint_step",
           "hydro_prim_to_cons", "hydro_prim_to_cons_adjoint", "hydro_run", "hydro_autotune", "hydro_get_tuning",
           "hydro_set_tuning", "hydro_get_class_tuning", "hydro_set_class_tuning", "hydro_get_error", "hydro_clear_error", "hydro_launch_count", "hydro_status_string",
           "hydro_step_batched_noalloc")


class HydroError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, status_string(status), status))


class hydro_config(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("rho_floor", ctypes.c_double),
                ("p_floor", ctypes.c_double), ("limiter", ctypes.c_int), ("precision", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class hydro_patch(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p * 5), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ng", ctypes.c_int), ("sy", ctypes.c_longlong), ("sz", ctypes.c_longlong), ("dx", ctypes.c_double),
                ("level", ctypes.c_int)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhydro.so is not built; run paper_1412_0934_gb300.build.build() "
                               "(or __graft_entry__.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        PP = ctypes.POINTER(hydro_patch)
        L.hydro_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(hydro_config)]
        L.hydro_finalize.argtypes = [vp]
        L.hydro_cfl_dt.argtypes = [vp, PP, i, vp]
        L.hydro_step.argtypes = [vp, PP, PP, i, vp, vp]
        L.hydro_step_host.argtypes = [vp, PP, PP, vp, vp]
        L.hydro_step_octs.argtypes = [vp, vp * 5, vp * 5, ll, d, vp]
        L.hydro_step_octs_level.argtypes = [vp, PP, vp, ll, vp * 5, vp]
        L.hydro_octs_build.argtypes = [vp, vp, i, ctypes.POINTER(ctypes.c_int), vp, vp]
        L.hydro_mhd_step.argtypes = [vp, vp * 9, vp * 9, i, i, i, d, vp, vp]
        L.hydro_mhd_cfl_dt.argtypes = [vp, vp * 9, i, i, i, d, vp]
        MP = ctypes.POINTER(hydro_mhd_patch)
        L.hydro_mhd_step_patches.argtypes = [vp, MP, MP, i, vp, vp]
        L.hydro_mhd_cfl_patches.argtypes = [vp, MP, i, vp]
        L.hydro_step_octs_table.argtypes = [vp, vp * 5, vp * 5, i, vp, vp, ll, d, vp]
        L.hydro_fill_ghosts.argtypes = [vp, PP, PP, ctypes.POINTER(ctypes.c_int), i]
        L.hydro_fill_ghosts_time.argtypes = [vp, PP, PP, d, PP, ctypes.POINTER(ctypes.c_int), i]
        L.hydro_exchange_ghosts.argtypes = [vp, PP, ctypes.POINTER(ctypes.c_int), i, ctypes.POINTER(ctypes.c_int)]
        IP = ctypes.POINTER(ctypes.c_int)
        L.hydro_patch_fluxes.argtypes = [vp, PP, i, vp, ctypes.POINTER(vp), i]
        L.hydro_level_fluxes.argtypes = [vp, PP, IP, IP, i, vp, ctypes.POINTER(vp), i]
        L.hydro_reflux.argtypes = [vp, PP, IP, IP, i, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.hydro_average_down.argtypes = [vp, PP, PP, IP, i]
        L.hydro_adjoint_step.argtypes = [vp, PP, vp, PP, PP, i]
        L.hydro_prim_to_cons.argtypes = [vp, PP, PP, i]
        L.hydro_prim_to_cons_adjoint.argtypes = [vp, PP, PP, PP, i]
        L.hydro_run.argtypes = [vp, PP, PP, i, vp, i]
        L.hydro_autotune.argtypes = [vp, PP, PP, i, vp, ctypes.c_char_p]
        L.hydro_get_tuning.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.hydro_set_tuning.argtypes = [vp, i, i]
        L.hydro_get_class_tuning.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.hydro_set_class_tuning.argtypes = [vp, i, i, i]
        L.hydro_get_error.argtypes = [vp, ctypes.POINTER(ctypes.c_uint)]
        L.hydro_clear_error.argtypes = [vp]
        L.hydro_launch_count.argtypes = [vp, ctypes.POINTER(ll)]
        L.hydro_step_batched_noalloc.argtypes = [ctypes.POINTER(hydro_config), PP, PP, i, vp, vp, vp]
        L.hydro_status_string.argtypes = [i]
        L.hydro_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def status_string(status):
    return lib().hydro_status_string(int(status)).decode()


def hydro_status_string(status):
    return status_string(status)


def _check(rc, what):
    if rc != HYDRO_OK:
        raise HydroError(rc, what)


class hydro_mhd_patch(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p * 9), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ng", ctypes.c_int), ("sy", ctypes.c_longlong), ("sz", ctypes.c_longlong), ("dx", ctypes.c_double),
                ("level", ctypes.c_int)]


class MhdPatch:
    """A hydro_mhd_patch plus the tensors it points into: fields (9, nz+2ng, ny+2ng, nx+2ng)."""

    def __init__(self, fields, ng, dx, level=0):
        fs = [fields[v] for v in range(9)] if isinstance(fields, torch.Tensor) else list(fields)
        if len(fs) != 9:
            raise ValueError("expected nine MHD fields")
        for f in fs:
            if not f.is_cuda or f.dim() != 3 or f.stride(2) != 1:
                raise ValueError("MHD patch fields must be 3D CUDA tensors with unit x stride")
            if f.shape != fs[0].shape or f.stride() != fs[0].stride() or f.dtype != fs[0].dtype:
                raise ValueError("fields must share shape, strides and dtype")
        Z, Y, X = fs[0].shape
        self.tensors = fs
        self.dtype = fs[0].dtype
        self.c = hydro_mhd_patch()
        for v in range(9):
            self.c.U[v] = fs[v].data_ptr()
        self.c.nx, self.c.ny, self.c.nz = X - 2 * ng, Y - 2 * ng, Z - 2 * ng
        self.c.ng = ng
        self.c.sy = fs[0].stride(1)
        self.c.sz = fs[0].stride(0)
        self.c.dx = float(dx)
        self.c.level = int(level)


def _mhd_parray(patches):
    patches = list(patches)
    return (hydro_mhd_patch * len(patches))(*[p.c for p in patches]), len(patches)


class Patch:
    """A hydro_patch plus the tensors it points into (kept alive while the patch is)."""

    def __init__(self, fields, ng, dx, level=0, host=False):
        if isinstance(fields, torch.Tensor):
            if fields.dim() != 4 or fields.shape[0] != 5:
                raise ValueError("expected a (5, nz, ny, nx) tensor")
            fs = [fields[v] for v in range(5)]
        else:
            fs = list(fields)
            if len(fs) != 5:
                raise ValueError("expected five field tensors")
        for f in fs:
            if f.is_cuda == host:
                raise ValueError("patch fields must be %s tensors" % ("host (CPU)" if host else "CUDA"))
            if f.dim() != 3 or f.stride(2) != 1:
                raise ValueError("each field must be 3D with unit x stride")
            if f.shape != fs[0].shape or f.stride() != fs[0].stride() or f.dtype != fs[0].dtype:
                raise ValueError("fields must share shape, strides and dtype")
        Z, Y, X = fs[0].shape
        self.tensors = fs
        self.dtype = fs[0].dtype
        self.c = hydro_patch()
        for v in range(5):
            self.c.U[v] = fs[v].data_ptr()
        self.c.nx, self.c.ny, self.c.nz = X - 2 * ng, Y - 2 * ng, Z - 2 * ng
        self.c.ng = ng
        self.c.sy = fs[0].stride(1)
        self.c.sz = fs[0].stride(0)
        self.c.dx = float(dx)
        self.c.level = int(level)


def patch(fields, ng, dx, level=0):
    return Patch(fields, ng, dx, level)


def host_patch(fields, dx):
    """A periodic box (ng = 0) in host memory, for hydro_step_host (page-locked tensors overlap)."""
    return Patch(fields, 0, dx, host=True)


def _parray(patches):
    patches = [patches] if isinstance(patches, Patch) else list(patches)
    arr = (hydro_patch * len(patches))(*[p.c for p in patches])
    return arr, len(patches)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


def _f64(t, n, what):
    """Pointer to a CUDA float64 tensor of at least n elements (the time-step arrays), or None."""
    if t is None:
        return None
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() < n:
        raise ValueError("%s must be a contiguous float64 CUDA tensor of at least %d elements" % (what, n))
    return _ptr(t)


def _dtypes(obj):
    if isinstance(obj, (Patch, MhdPatch, torch.Tensor)):
        yield obj.dtype
    elif isinstance(obj, (list, tuple)):
        for o in obj:
            yield from _dtypes(o)


def _same_dtype(ctx, *objs):
    """The fields and registers a call reads or writes must hold the context's element type: the
    library addresses them with it (double, or float for HYDRO_FP32)."""
    for o in objs:
        for dt in _dtypes(o):
            if dt != ctx.dtype:
                raise ValueError("the context works on %s data; got %s" % (ctx.dtype, dt))


class Context:
    """An open hydro_ctx (create with hydro_init, release with hydro_finalize)."""

    def __init__(self, handle, cfg):
        self.handle = handle
        self.cfg = cfg

    @property
    def precision(self):
        return self.cfg.precision

    @property
    def dtype(self):
        return torch.float32 if self.cfg.precision == HYDRO_FP32 else torch.float64

    def __del__(self):
        try:
            if self.handle:
                lib().hydro_finalize(self.handle)
                self.handle = None
        except Exception:
            pass


def hydro_init(gamma=5.0 / 3.0, cfl=0.8, rho_floor=1e-10, p_floor=1e-14, limiter="minmod", precision="fp64",
               stream=None):
    """Open a context on the current device; all calls go to `stream` (default: torch's current stream)."""
    cfg = hydro_config()
    cfg.gamma, cfg.cfl, cfg.rho_floor, cfg.p_floor = gamma, cfl, rho_floor, p_floor
    cfg.limiter = LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if stream is None:
        stream = torch.cuda.current_stream()
    cfg.cuda_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    h = ctypes.c_void_p()
    _check(lib().hydro_init(ctypes.byref(h), ctypes.byref(cfg)), "hydro_init")
    return Context(h, cfg)


def hydro_finalize(ctx):
    if ctx.handle:
        _check(lib().hydro_finalize(ctx.handle), "hydro_finalize")
        ctx.handle = None


def hydro_cfl_dt(ctx, patches, dt_out):
    _same_dtype(ctx, patches)
    arr, n = _parray(patches)
    _check(lib().hydro_cfl_dt(ctx.handle, arr, n, _f64(dt_out, n, "dt_out")), "hydro_cfl_dt")


def hydro_step(ctx, inp, out, dt, dt_next=None):
    a, n = _parray(inp)
    b, m = _parray(out)
    if n != m:
        raise ValueError("in and out patch counts differ")
    _same_dtype(ctx, inp, out)
    _check(lib().hydro_step(ctx.handle, a, b, n, _f64(dt, n, "dt"), _f64(dt_next, n, "dt_next")), "hydro_step")


def hydro_step_host(ctx, inp, out, dt, dt_next=None):
    """One step of a host-resident periodic box (host_patch in / out; dt, dt_next CUDA tensors)."""
    _same_dtype(ctx, inp, out)
    _check(lib().hydro_step_host(ctx.handle, ctypes.byref(inp.c), ctypes.byref(out.c), _f64(dt, 1, "dt"),
                                 _f64(dt_next, 1, "dt_next")), "hydro_step_host")


def hydro_fill_ghosts(ctx, coarse, fine, origins):
    """Fill the ghost layers of the fine patches (list of Patch, ng = 2) from the periodic coarse
    Patch; origins: (x, y, z) fine-level index of each patch's first interior cell."""
    f, n = _parray(fine)
    o = (ctypes.c_int * (3 * n))(*[int(v) for xyz in origins for v in xyz])
    if len(o) != 3 * n:
        raise ValueError("one (x, y, z) origin per patch")
    _same_dtype(ctx, coarse, fine)
    _check(lib().hydro_fill_ghosts(ctx.handle, ctypes.byref(coarse.c), f, o, n), "hydro_fill_ghosts")


def hydro_fill_ghosts_time(ctx, coarse_old, coarse_new, theta, fine, origins):
    """hydro_fill_ghosts from the coarse level at the fraction theta of its step:
    (1 - theta) coarse_old + theta coarse_new, then prolonged."""
    f, n = _parray(fine)
    o = (ctypes.c_int * (3 * n))(*[int(v) for xyz in origins for v in xyz])
    if len(o) != 3 * n:
        raise ValueError("one (x, y, z) origin per patch")
    _same_dtype(ctx, coarse_old, coarse_new, fine)
    _check(lib().hydro_fill_ghosts_time(ctx.handle, ctypes.byref(coarse_old.c), ctypes.byref(coarse_new.c),
                                        float(theta), f, o, n), "hydro_fill_ghosts_time")


def hydro_exchange_ghosts(ctx, fine, origins, period):
    """Ghosts of the patches (list of Patch, ng = 2) covered by a same-level interior take its
    values; origins: first interior cell (x, y, z) per patch; period: (x, y, z) of the level."""
    f, n = _parray(fine)
    o = (ctypes.c_int * (3 * n))(*[int(v) for xyz in origins for v in xyz])
    if len(o) != 3 * n:
        raise ValueError("one (x, y, z) origin per patch")
    per = (ctypes.c_int * 3)(*[int(v) for v in period])
    _same_dtype(ctx, fine)
    _check(lib().hydro_exchange_ghosts(ctx.handle, f, o, n, per), "hydro_exchange_ghosts")


def register_size(nx, ny, nz):
    """Elements per field of a flux register of an nx x ny x nz box."""
    return 2 * (ny * nz + nx * nz + nx * ny)


def _ints(rows):
    flat = [int(v) for r in rows for v in r]
    return (ctypes.c_int * len(flat))(*flat)


def _ptrs(tensors):
    return (ctypes.c_void_p * len(tensors))(*[_ptr(t) for t in tensors])


def hydro_patch_fluxes(ctx, patches, dt, registers, accumulate=False):
    """registers[p]: CUDA tensor of 5 * register_size(...) elements of the storage type."""
    a, n = _parray(patches)
    if len(registers) != n:
        raise ValueError("one register per patch")
    _same_dtype(ctx, patches, registers)
    _check(lib().hydro_patch_fluxes(ctx.handle, a, n, _f64(dt, n, "dt"), _ptrs(registers), int(bool(accumulate))),
           "hydro_patch_fluxes")


def hydro_level_fluxes(ctx, level, box_origins, box_dims, dt, registers, accumulate=False):
    n = len(box_origins)
    if len(box_dims) != n or len(registers) != n:
        raise ValueError("one origin, size and register per box")
    _same_dtype(ctx, level, registers)
    _check(lib().hydro_level_fluxes(ctx.handle, ctypes.byref(level.c), _ints(box_origins), _ints(box_dims), n,
                                    _f64(dt, 1, "dt"), _ptrs(registers), int(bool(accumulate))), "hydro_level_fluxes")


def hydro_reflux(ctx, coarse, box_origins, box_dims, coarse_registers, fine_registers):
    n = len(box_origins)
    if len(box_dims) != n or len(coarse_registers) != n or len(fine_registers) != n:
        raise ValueError("one origin, size and pair of registers per box")
    _same_dtype(ctx, coarse, coarse_registers, fine_registers)
    _check(lib().hydro_reflux(ctx.handle, ctypes.byref(coarse.c), _ints(box_origins), _ints(box_dims), n,
                              _ptrs(coarse_registers), _ptrs(fine_registers)), "hydro_reflux")


def hydro_average_down(ctx, coarse, fine, origins):
    f, n = _parray(fine)
    if len(origins) != n:
        raise ValueError("one origin per patch")
    _same_dtype(ctx, coarse, fine)
    _check(lib().hydro_average_down(ctx.handle, ctypes.byref(coarse.c), f, _ints(origins), n), "hydro_average_down")


def hydro_step_octs_level(ctx, level, origins, out, dt):
    """level: periodic Patch of the level grid; origins: (G, 3) int32 CUDA tensor (x, y, z);
    out: (5, G, 2, 2, 2)."""
    if origins.dtype != torch.int32 or not origins.is_contiguous() or origins.dim() != 2 or origins.shape[1] != 3:
        raise ValueError("origins must be a contiguous (G, 3) int32 tensor")
    o = (ctypes.c_void_p * 5)(*[_ptr(out[v]) for v in range(5)])
    for v in range(5):
        if not out[v].is_contiguous():
            raise ValueError("oct arrays must be contiguous per field")
    _same_dtype(ctx, level, out)
    _check(lib().hydro_step_octs_level(ctx.handle, ctypes.byref(level.c), _ptr(origins), origins.shape[0], o,
                                       _f64(dt, 1, "dt")), "hydro_step_octs_level")


def _int_tensor(t, what, cols=None):
    if t.dtype != torch.int32 or not t.is_contiguous() or (cols and (t.dim() != 2 or t.shape[1] != cols)):
        raise ValueError("%s must be a contiguous int32 tensor%s" % (what, " of shape (n, %d)" % cols if cols else ""))


def hydro_octs_build(ctx, pos, dims, order, nbr=None):
    """pos: (n, 3) int32 CUDA tensor of oct coordinates (X, Y, Z); dims: 3 ints (octs per axis);
    order: (n,) int32 out, the Morton order; nbr: None or (n, 27) int32 out, the neighbour table."""
    _int_tensor(pos, "pos", 3)
    _int_tensor(order, "order")
    if nbr is not None:
        _int_tensor(nbr, "nbr", 27)
    d = (ctypes.c_int * 3)(*[int(v) for v in dims])
    _check(lib().hydro_octs_build(ctx.handle, _ptr(pos), pos.shape[0], d, _ptr(order),
                                  _ptr(nbr) if nbr is not None else None), "hydro_octs_build")


def hydro_step_octs_table(ctx, U, out, nbr, octs, dx, dt):
    """U, out: (5, noct, 8) oct-major level (or 5 tensors of (noct, 8)); nbr: (noct, 27) int32;
    octs: (G,) int32 list of the octs to step; their cells of out receive U^{n+1}."""
    _int_tensor(nbr, "nbr", 27)
    _int_tensor(octs, "octs")
    i = (ctypes.c_void_p * 5)(*[_ptr(U[v]) for v in range(5)])
    o = (ctypes.c_void_p * 5)(*[_ptr(out[v]) for v in range(5)])
    for v in range(5):
        if not U[v].is_contiguous() or not out[v].is_contiguous():
            raise ValueError("oct arrays must be contiguous per field")
    _same_dtype(ctx, U, out)
    _check(lib().hydro_step_octs_table(ctx.handle, i, o, nbr.shape[0], _ptr(nbr), _ptr(octs), octs.shape[0],
                                       float(dx), _f64(dt, 1, "dt")), "hydro_step_octs_table")


def _mhd_fields(U):
    if len(U) != 9:
        raise ValueError("MHD state: nine fields (rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi)")
    for v in range(9):
        if not U[v].is_contiguous() or U[v].shape != U[0].shape or U[v].dim() != 3:
            raise ValueError("MHD fields must be contiguous (nz, ny, nx) tensors of one shape")
    nz, ny, nx = U[0].shape
    return (ctypes.c_void_p * 9)(*[_ptr(U[v]) for v in range(9)]), nx, ny, nz


def hydro_mhd_step(ctx, U, out, dx, dt, dt_next=None):
    """U, out: (9, nz, ny, nx) tensors (or 9 tensors) of a periodic box; dt: device double."""
    a, nx, ny, nz = _mhd_fields(U)
    b, *_ = _mhd_fields(out)
    _same_dtype(ctx, U, out)
    _check(lib().hydro_mhd_step(ctx.handle, a, b, nx, ny, nz, float(dx), _f64(dt, 1, "dt"),
                                _f64(dt_next, 1, "dt_next")), "hydro_mhd_step")


def hydro_mhd_step_patches(ctx, inp, out, dt, dt_next=None):
    """inp, out: lists of MhdPatch (ng 2 in; 0 or 2 out); dt: (npatch,) device doubles."""
    a, n = _mhd_parray(inp)
    b, m = _mhd_parray(out)
    if m != n:
        raise ValueError("one output patch per input patch")
    _same_dtype(ctx, inp, out)
    _check(lib().hydro_mhd_step_patches(ctx.handle, a, b, n, _f64(dt, n, "dt"), _f64(dt_next, n, "dt_next")),
           "hydro_mhd_step_patches")


def hydro_mhd_cfl_patches(ctx, patches, dt):
    a, n = _mhd_parray(patches)
    _same_dtype(ctx, patches)
    _check(lib().hydro_mhd_cfl_patches(ctx.handle, a, n, _f64(dt, n, "dt")), "hydro_mhd_cfl_patches")


def hydro_mhd_cfl_dt(ctx, U, dx, dt):
    a, nx, ny, nz = _mhd_fields(U)
    _same_dtype(ctx, U)
    _check(lib().hydro_mhd_cfl_dt(ctx.handle, a, nx, ny, nz, float(dx), _f64(dt, 1, "dt")), "hydro_mhd_cfl_dt")


def hydro_step_octs(ctx, gathered, out, dx, dt):
    """gathered: (5, G, 6, 6, 6) tensor (or 5 tensors); out: (5, G, 2, 2, 2)."""
    g = (ctypes.c_void_p * 5)(*[_ptr(gathered[v]) for v in range(5)])
    o = (ctypes.c_void_p * 5)(*[_ptr(out[v]) for v in range(5)])
    for v in range(5):
        if not gathered[v].is_contiguous() or not out[v].is_contiguous():
            raise ValueError("oct arrays must be contiguous per field")
    G = gathered[0].shape[0]
    _same_dtype(ctx, gathered, out)
    _check(lib().hydro_step_octs(ctx.handle, g, o, G, float(dx), _f64(dt, 1, "dt")), "hydro_step_octs")


def hydro_adjoint_step(ctx, U_n, dt, lam_np1, lam_n):
    a, n = _parray(U_n)
    b, _ = _parray(lam_np1)
    c, _ = _parray(lam_n)
    _same_dtype(ctx, U_n, lam_np1, lam_n)
    _check(lib().hydro_adjoint_step(ctx.handle, a, _f64(dt, n, "dt"), b, c, n), "hydro_adjoint_step")


def hydro_prim_to_cons(ctx, W, U):
    a, n = _parray(W)
    b, _ = _parray(U)
    _same_dtype(ctx, W, U)
    _check(lib().hydro_prim_to_cons(ctx.handle, a, b, n), "hydro_prim_to_cons")


def hydro_prim_to_cons_adjoint(ctx, W, lamU, lamW):
    a, n = _parray(W)
    b, _ = _parray(lamU)
    c, _ = _parray(lamW)
    _same_dtype(ctx, W, lamU, lamW)
    _check(lib().hydro_prim_to_cons_adjoint(ctx.handle, a, b, c, n), "hydro_prim_to_cons_adjoint")


def hydro_run(ctx, a, b, nsteps, dt_hist, use_graph=True):
    pa, _ = _parray(a)
    pb, _ = _parray(b)
    _same_dtype(ctx, a, b)
    _check(lib().hydro_run(ctx.handle, pa, pb, int(nsteps), _f64(dt_hist, int(nsteps) + 1, "dt_hist"),
                           1 if use_graph else 0), "hydro_run")


def hydro_autotune(ctx, inp, out, dt, cache_path=None):
    a, n = _parray(inp)
    b, _ = _parray(out)
    cp = cache_path.encode() if cache_path else None
    _same_dtype(ctx, inp, out)
    _check(lib().hydro_autotune(ctx.handle, a, b, n, _f64(dt, n, "dt"), cp), "hydro_autotune")


def hydro_get_tuning(ctx):
    t, z = ctypes.c_int(), ctypes.c_int()
    _check(lib().hydro_get_tuning(ctx.handle, ctypes.byref(t), ctypes.byref(z)), "hydro_get_tuning")
    return t.value, z.value


def hydro_set_tuning(ctx, tile_id, zchunk):
    _check(lib().hydro_set_tuning(ctx.handle, int(tile_id), int(zchunk)), "hydro_set_tuning")


def hydro_get_class_tuning(ctx, patch_class):
    t, z = ctypes.c_int(), ctypes.c_int()
    _check(lib().hydro_get_class_tuning(ctx.handle, int(patch_class), ctypes.byref(t), ctypes.byref(z)),
           "hydro_get_class_tuning")
    return t.value, z.value


def hydro_set_class_tuning(ctx, patch_class, tile_id, zchunk=0):
    """tile_id -1: the class steps with the context's tuning (hydro_set_tuning's)."""
    _check(lib().hydro_set_class_tuning(ctx.handle, int(patch_class), int(tile_id), int(zchunk)),
           "hydro_set_class_tuning")


def hydro_get_error(ctx):
    """(status, bits): synchronises the context's stream."""
    bits = ctypes.c_uint()
    rc = lib().hydro_get_error(ctx.handle, ctypes.byref(bits))
    if rc not in (HYDRO_OK, HYDRO_ERR_UNPHYSICAL):
        raise HydroError(rc, "hydro_get_error")
    return rc, bits.value


def hydro_clear_error(ctx):
    _check(lib().hydro_clear_error(ctx.handle), "hydro_clear_error")


def hydro_step_batched_noalloc(cfg, inp, out, npatch, dt, dt_next=None, error_bits=None):
    """The batched step without a context and without any device allocation (see include/hydro.h).
    cfg: a hydro_config; inp, out: ctypes arrays of hydro_patch; dt, dt_next, error_bits: CUDA
    tensors (or None).  Returns the status code."""
    return lib().hydro_step_batched_noalloc(ctypes.byref(cfg), inp, out, int(npatch), _ptr(dt), _ptr(dt_next),
                                            _ptr(error_bits))


def hydro_launch_count(ctx):
    n = ctypes.c_longlong()
    _check(lib().hydro_launch_count(ctx.handle, ctypes.byref(n)), "hydro_launch_count")
    return n.value
