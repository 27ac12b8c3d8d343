"""Build libhydro.so (the sm_103a CUDA library behind include/hydro.h) in-tree with nvcc.

Each translation unit compiles in parallel for one target only (sm_103a); the objects are
linked into paper_1412_0934_gb300/libhydro.so.  Rebuilds only what changed.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhydro.so")
INCLUDE = os.path.join(ROOT, "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC,
         "--expt-relaxed-constexpr"]
SOURCES = ["hydro_api.cu", "worklist.cu", "kernels_f64.cu", "kernels_f32.cu", "kernels_mixed.cu", "kernels_df.cu", "noalloc.cu",
           "ghosts.cu", "octs_build.cu", "mhd.cu"]


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def _compile(src, obj, verbose, extra):
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return r.stderr


def build(force=False, verbose=False, ptxas_info=False, checked=False):
    """Build libhydro.so, or with checked=True the bounds-checked variant libhydro_checked.so (every
    global index of the step kernels tested against its array's extent: HYDRO_EBIT_OOB), loaded
    instead of the default library when the environment variable HYDRO_LIBRARY names it."""
    bdir = BUILD + ("_checked" if checked else "")
    lib = LIB.replace("libhydro.so", "libhydro_checked.so") if checked else LIB
    os.makedirs(bdir, exist_ok=True)
    hdr_time = _newest(_headers())
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DHYDRO_CHECK_BOUNDS"] if checked else [])
    jobs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or ptxas_info or not os.path.exists(obj) or os.path.getmtime(obj) < max(
                hdr_time, os.path.getmtime(os.path.join(CSRC, src))):
            jobs.append((src, obj))
    logs = {}
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            futs = {ex.submit(_compile, s, o, verbose, extra): s for s, o in jobs}
            for f in concurrent.futures.as_completed(futs):
                logs[futs[f]] = f.result()
    if jobs or force or not os.path.exists(lib):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib, logs


if __name__ == "__main__":
    _, logs = build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    for k, v in logs.items():
        if v.strip():
            print("==", k)
            print(v)
