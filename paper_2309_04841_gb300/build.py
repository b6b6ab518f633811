"""Build ``libqaoa.so`` (the C-ABI library) in-tree for sm_103a.

Each CUDA translation unit is compiled by its own nvcc process (in parallel),
then linked into ``paper_2309_04841_gb300/libqaoa.so`` against the shared
CUDA runtime, so the process shares one runtime with PyTorch.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqaoa.so")
# (source, object, extra flags): the TMA kernels are compiled once per cost
# element width (4 bytes: int32 / float32; 2 bytes: uint16), in parallel.
UNITS = [("api.cu", "api.o", []), ("pass_kernels.cu", "pass_kernels.o", []),
         ("small_kernels.cu", "small_kernels.o", []), ("cost_kernels.cu", "cost_kernels.o", []),
         ("profile.cu", "profile.o", []), ("tma_kernels.cu", "tma_kernels.o", []),
         ("tma_kernels.cu", "tma_kernels_u16.o", ["-DQAOA_TMA_CW=2"]),
         ("noalloc.cu", "noalloc.o", []), ("serve.cu", "serve.o", []),
         ("xy_kernels.cu", "xy_kernels.o", [])]
SOURCES = sorted({u[0] for u in UNITS})
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqaoa.so")
    return path


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "qaoa.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(unit, verbose):
    src, obj_name, extra = unit
    obj = os.path.join(BUILD, obj_name)
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *extra,
           "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


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


def build(force=False, verbose=False):
    """Compile and link; returns the library path.  Rebuilds when any source
    is newer than the library."""
    if (not force and os.path.exists(LIB) and _native(LIB)
            and os.path.getmtime(LIB) >= _deps()):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda u: _compile(u, verbose), UNITS))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
