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
