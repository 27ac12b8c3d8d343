"""CPU checks of the boundary: the library builds, loads without a GPU, and exports every entry
point include/hydro.h declares; the binding rejects bad calls before reaching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(hydro_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1412_0934_gb300 import build
    path, _ = build.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hydro_init", "hydro_step", "hydro_cfl_dt", "hydro_adjoint_step", "hydro_step_octs", "hydro_finalize",
              "hydro_get_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_lists_every_export(libpath):
    import paper_1412_0934_gb300 as hy
    assert set(hy.EXPORTS) == declared_functions()


def test_status_strings(libpath):
    import paper_1412_0934_gb300 as hy
    assert hy.status_string(hy.HYDRO_ERR_ARG) == "invalid argument"
    assert hy.status_string(0) == "ok"


def test_init_rejects_bad_config_without_gpu(libpath):
    import paper_1412_0934_gb300 as hy
    L = hy.lib()
    for bad in [dict(gamma=1.0), dict(cfl=0.0), dict(cfl=1.5), dict(rho_floor=-1.0), dict(limiter=7),
                dict(precision=9)]:
        cfg = hy.hydro_config()
        cfg.gamma, cfg.cfl, cfg.rho_floor, cfg.p_floor, cfg.limiter, cfg.precision = 5 / 3, 0.8, 1e-10, 1e-14, 0, 0
        for k, v in bad.items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        assert L.hydro_init(ctypes.byref(h), ctypes.byref(cfg)) == hy.HYDRO_ERR_ARG
        assert not h.value
    assert L.hydro_init(None, None) == hy.HYDRO_ERR_ARG


def test_null_context_calls_are_argument_errors(libpath):
    """Every entry point called with a NULL context (or config), NULL pointers and zero counts
    returns HYDRO_ERR_ARG from its host-side checks, before any CUDA call (finalize of NULL is a
    no-op; the status string is static)."""
    import paper_1412_0934_gb300 as hy
    L = hy.lib()
    scalars = (ctypes.c_int, ctypes.c_uint, ctypes.c_long, ctypes.c_longlong, ctypes.c_size_t, ctypes.c_double,
               ctypes.c_float)
    results = {}
    for name in sorted(hy.EXPORTS):
        f = getattr(L, name)
        assert f.argtypes is not None, name
        args = []
        for t in f.argtypes:
            if t in scalars:
                args.append(0)
            elif isinstance(t, type) and issubclass(t, ctypes.Array):
                args.append(t())
            else:
                args.append(None)
        results[name] = f(*args)
    assert results.pop("hydro_finalize") == hy.HYDRO_OK
    assert results.pop("hydro_status_string") == b"ok"
    bad = {k: v for k, v in results.items() if v != hy.HYDRO_ERR_ARG}
    assert not bad, bad


def _fake_patch(hy, base, n, ng, dx=0.01):
    """A hydro_patch over made-up, aligned, non-overlapping addresses: only host-side checks read it."""
    nx, ny, nz = n
    p = hy.hydro_patch()
    sy, sz = nx + 2 * ng, (nx + 2 * ng) * (ny + 2 * ng)
    field = (nz + 2 * ng) * sz * 8
    for v in range(5):
        p.U[v] = base + v * ((field + 4095) // 4096 * 4096)
    p.nx, p.ny, p.nz, p.ng, p.sy, p.sz, p.dx, p.level = nx, ny, nz, ng, sy, sz, dx, 0
    return p


def test_noalloc_host_checks_without_gpu(libpath):
    """hydro_step_batched_noalloc refuses, on the host and before any CUDA call: a missing error
    word, more tiles than its static work-list holds (262144 of 16 x 16 x 32), more than 4096
    patches, and ghost widths hydro_step refuses (a batched input patch without two ghost layers)."""
    import paper_1412_0934_gb300 as hy
    L = hy.lib()
    cfg = hy.hydro_config()
    cfg.gamma, cfg.cfl, cfg.rho_floor, cfg.p_floor, cfg.limiter, cfg.precision = 5 / 3, 0.8, 1e-10, 1e-14, 0, 0
    dt, dn, err = 1 << 40, 2 << 40, 3 << 40  # never dereferenced: every call below fails its host checks

    def call(ins, outs, err_word=err):
        a = (hy.hydro_patch * len(ins))(*ins)
        b = (hy.hydro_patch * len(outs))(*outs)
        return L.hydro_step_batched_noalloc(ctypes.byref(cfg), a, b, len(ins), dt, dn, err_word)

    small_in = [_fake_patch(hy, (4 + 2 * k) << 32, (8, 8, 8), 2) for k in range(3)]
    small_out = [_fake_patch(hy, (5 + 2 * k) << 32, (8, 8, 8), 2) for k in range(3)]
    assert call(small_in, small_out, None) == hy.HYDRO_ERR_ARG
    # 2048 x 2048 x 1024 interior: 128 x 128 x 32 = 524288 tiles
    huge_in, huge_out = _fake_patch(hy, 1 << 44, (2048, 2048, 1024), 2), _fake_patch(hy, 1 << 45, (2048, 2048, 1024), 2)
    assert call([huge_in], [huge_out]) == hy.HYDRO_ERR_ARG
    many_in = [_fake_patch(hy, (1 << 36) + k * (1 << 24), (4, 4, 4), 2) for k in range(4097)]
    many_out = [_fake_patch(hy, (1 << 37) + k * (1 << 24), (4, 4, 4), 2) for k in range(4097)]
    assert call(many_in, many_out) == hy.HYDRO_ERR_ARG
    # a batch of periodic (ng = 0) inputs, and a 1-ghost-layer input, as hydro_step refuses them
    per_in = [_fake_patch(hy, (4 + 2 * k) << 32, (8, 8, 8), 0) for k in range(2)]
    per_out = [_fake_patch(hy, (5 + 2 * k) << 32, (8, 8, 8), 0) for k in range(2)]
    assert call(per_in, per_out) == hy.HYDRO_ERR_ARG
    one_in = [_fake_patch(hy, 4 << 32, (8, 8, 8), 1)]
    one_out = [_fake_patch(hy, 5 << 32, (8, 8, 8), 1)]
    assert call(one_in, one_out) == hy.HYDRO_ERR_ARG


def test_tile_shapes_agree_across_header_library_and_binding():
    """The binding's tile table, the header's HYDRO_NUM_TILES and the compiled shape table agree."""
    import paper_1412_0934_gb300 as hy
    hdr = open(os.path.join(ROOT, "include", "hydro.h")).read()
    assert int(re.search(r"#define HYDRO_NUM_TILES (\d+)", hdr).group(1)) == hy.NUM_TILES
    src = open(os.path.join(ROOT, "paper_1412_0934_gb300", "csrc", "internal.h")).read()
    xs = [int(v) for v in re.search(r"kTileX\[kNumTiles\] = \{([^}]*)\}", src).group(1).split(",")]
    ys = [int(v) for v in re.search(r"kTileY\[kNumTiles\] = \{([^}]*)\}", src).group(1).split(",")]
    assert tuple(zip(xs, ys)) == hy.TILE_SHAPES
    assert int(re.search(r"#define HYDRO_NUM_PATCH_CLASSES (\d+)", hdr).group(1)) == hy.NUM_PATCH_CLASSES
