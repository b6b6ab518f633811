"""Compile ``oracle/oracle.c`` into ``oracle/liboracle.so`` with plain gcc.

Test infrastructure: the oracle is the checker, not the product.  Flags keep
float64 arithmetic literal: no fast-math and no FMA contraction, so additions
happen exactly in the order the source states.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
# the same source with OpenMP: only the benchmark's all-core CPU figure
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def _native(path):
    """True if the ELF file at path was built for this machine's architecture."""
    import platform
    want = {"x86_64": 0x3E, "amd64": 0x3E, "aarch64": 0xB7, "arm64": 0xB7}.get(
        platform.machine().lower())
    try:
        with open(path, "rb") as fh:
            hdr = fh.read(20)
    except OSError:
        return False
    return len(hdr) == 20 and hdr[:4] == b"\x7fELF" and (want is None or hdr[18] == want)


def _build_one(lib, extra, force):
    if (not force and os.path.exists(lib) and _native(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(SRC)):
        return lib
    tmp = f"{lib}.{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", *extra, "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """The single-threaded oracle (the OpenMP pragmas are ignored)."""
    return _build_one(LIB, ["-Wno-unknown-pragmas"], force)


def build_omp(force: bool = False) -> str:
    """The same source compiled with OpenMP (benchmark CPU figure only)."""
    return _build_one(LIB_OMP, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_omp(force="--force" in sys.argv))
