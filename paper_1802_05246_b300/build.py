"""Build the in-tree CUDA library libhermite_b300.so for sm_103a with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libhermite_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source to an object file (in parallel, the kernel
    instantiations make some files slow) and link the shared library."""
    if not force and not _stale():
        return LIB
    import concurrent.futures
    import tempfile

    tmp = LIB + f".tmp{os.getpid()}"
    flags = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", *ARCH, "-I", os.path.join(HERE, "..", "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    with tempfile.TemporaryDirectory() as objdir:
        srcs = sources()
        objs = [os.path.join(objdir, os.path.basename(s) + ".o") for s in srcs]
        with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            for f in [ex.submit(subprocess.check_call, [NVCC, *flags, "-c", s, "-o", o]) for s, o in zip(srcs, objs)]:
                f.result()
        subprocess.check_call([NVCC, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
