"""Build the sm_103a shared libraries in-tree with nvcc.

libhc_gb300.so is the product. Its translation units compile in parallel and
link into one shared object next to this file: the 2D and 3D kernels per
precision, the batched sweep kernels, the mixed-radix kernels of grids that
are not powers of two, the host orchestration with the C ABI, and the
allocation-free transform.

libhc_gb300_check.so is the bounds-checked build. HC_CHECK=1 changes only the
host orchestration (hc_api.cu: guard zones after every workspace buffer, and
the scan). So it shares the kernel objects and recompiles that one unit.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libhc_gb300.so")
LIB_CHECK = os.path.join(HERE, "libhc_gb300_check.so")
BUILD_DIR = os.path.join(HERE, "_build")
CHECK_SOURCE = "hc_api.cu"   # the only unit HC_CHECK changes

SOURCES = ["hc_kernels_f32.cu", "hc_kernels_f64.cu", "hc_kernels_df.cu", "hc_kernels3d_f32.cu",
           "hc_kernels3d_f64.cu", "hc_kernels3d_df.cu", "hc_batch.cu", "hc_generic.cu", "hc_api.cu",
           "hc_noalloc.cu"]
HEADERS = ["hc_internal.cuh", "hc_kernels.cuh", "hc_kernels3d.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE] + ARCH


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "hc.h"),
                                                                   os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def _obj(src: str, check: bool = False) -> str:
    name = src.replace(".cu", "_check.o" if check else ".o")
    return os.path.join(BUILD_DIR, name)


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds both libraries (whichever is out of date) and returns the product's path."""
    want_lib = force or _stale(LIB)
    want_check = force or _stale(LIB_CHECK)
    if not (want_lib or want_check):
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    # the checked library links the product's kernel objects: compile them too if any is missing
    have_objs = all(os.path.exists(_obj(src)) for src in SOURCES)
    units = [(src, False) for src in SOURCES] if want_lib or not have_objs else []
    if want_check:
        units.append((CHECK_SOURCE, True))
    procs = []
    for src, check in units:
        cmd = [nvcc()] + NVCC_FLAGS + (["-DHC_CHECK=1"] if check else []) + \
            ["-c", os.path.join(CSRC, src), "-o", _obj(src, check)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    for lib, check in ((LIB, False), (LIB_CHECK, True)):
        if not (want_check if check else want_lib):
            continue
        objs = [_obj(src, check and src == CHECK_SOURCE) for src in SOURCES]
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.run([nvcc(), "-shared"] + ARCH + ["-o", tmp] + objs, check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
