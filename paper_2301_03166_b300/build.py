"""Builds libabft.so (all CUDA sources under csrc/) for sm_103a, in-tree.

Each source compiles to its own object (in parallel, into _build/ at the
repository root), then nvcc links them into one shared library."""
import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libabft.so")
OBJ = os.path.join(ROOT, "_build", "abft")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def headers():
    return glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def deps():
    return sources() + headers()


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in deps())


def _obj(src):
    return os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")


def _compile(src, force, verbose):
    o = _obj(src)
    hdr = max((os.path.getmtime(h) for h in headers()), default=0.0)
    if not force and os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(src), hdr):
        return o
    cmd = [NVCC, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", "-o", o, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    return o


def build(force=False, verbose=False):
    """Compile every .cu in csrc/ and link one shared library with nvcc."""
    if not force and not stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, verbose), srcs))
    subprocess.run([NVCC, *ARCH, "-shared", "-o", LIB, *objs], check=True)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
