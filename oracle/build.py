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


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB) and _native(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
