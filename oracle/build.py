"""Build the FP64 CPU oracle (test infrastructure) into oracle/_oracle.so with g++.

Compiled with -ffp-contract=off so that every operation is a separately rounded IEEE double
operation on both x86_64 and aarch64 hosts (gcc contracts to FMA by default on aarch64).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_oracle.so")
SOURCES = [os.path.join(HERE, "oracle_capi.cpp")]
HEADERS = [os.path.join(HERE, h) for h in ("euler_oracle.hpp", "scalars.hpp")]


def _stale():
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(p) > t for p in SOURCES + HEADERS)


def command(sources, out):
    """The g++ command line that builds the oracle library `out` from `sources`."""
    return ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
            "-shared", "-fPIC", "-o", out] + list(sources)


def build(force=False, verbose=False):
    if not force and not _stale():
        return SO
    tmp = SO + ".tmp%d" % os.getpid()
    cmd = command(SOURCES, tmp)
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
