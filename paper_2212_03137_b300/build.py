"""Build the CUDA library ``libqhp.so`` in-tree for sm_103a (B300).

Usage: ``python -m paper_2212_03137_b300.build`` (or ``build()`` from Python).
The library is a plain C-ABI shared object; nothing here depends on torch.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libqhp.so")
LIB_CHECK = os.path.join(HERE, "libqhp_check.so")
SOURCES = ["capi.cu", "modes.cu", "neighbor.cu", "forces.cu", "qtb.cu", "noalloc.cu", "inspect.cu", "grad.cu", "batch.cu", "bar.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None, check: bool = False) -> str:
    """Compile every source to an object in parallel (each is a self-contained translation
    unit: no device code crosses files), then link the shared library.  check = True builds
    the bounds-checked variant libqhp_check.so (-DQHP_CHECK: indices read from device data
    are tested before use and reported as QHP_ERR_BOUNDS)."""
    from concurrent.futures import ThreadPoolExecutor

    lib = LIB_CHECK if check else LIB
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, "qhp_internal.cuh"), os.path.join(HERE, "..", "include", "qhp.h")]
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in deps):
            return lib
    objdir = os.path.join(HERE, "_build_check" if check else "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2", *(["-DQHP_CHECK"] if check else []),
             *(extra or [])]
    if verbose:
        flags.insert(0, "-Xptxas=-v")

    def compile_one(src: str):
        obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc(), *flags, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        return obj, cmd, res

    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, srcs))
    for obj, cmd, res in results:
        if verbose:
            print(" ".join(cmd))
            sys.stderr.write(res.stderr)
        if res.returncode != 0:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError(f"nvcc failed compiling {os.path.basename(obj)}")
    link = [nvcc(), *ARCH, "-shared", "-o", lib, *(o for o, _, _ in results), "-lcudart"]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError(f"nvcc failed linking {os.path.basename(lib)}")
    return lib


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, force=True)
    print(LIB)
