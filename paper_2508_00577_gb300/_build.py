"""Compile the CUDA sources of the package into an in-tree shared library.

nvcc, one -gencode for sm_103a, translation units compiled in parallel; the
FP64 stage kernels are compiled with --fmad=false so that their rounding
order is exactly the order written in the source.  build(bounds_check=True)
makes the bounds-checked variant libevlbm_bc.so (-DEVLBM_BOUNDS_CHECK: the
fused kernels count and skip out-of-range indices instead of using them).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libevlbm.so")
BUILD_BC = os.path.join(HERE, "_build_bc")
LIB_BC = os.path.join(HERE, "libevlbm_bc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-I", os.path.join(HERE, "..", "include")]
# Per-file extra flags.
EXTRA = {"ref_f64.cu": ["--fmad=false"], "noalloc.cu": ["--fmad=false"]}


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, bounds_check: bool = False) -> str:
    build_dir, lib_path = (BUILD_BC, LIB_BC) if bounds_check else (BUILD, LIB)
    defines = ["-DEVLBM_BOUNDS_CHECK"] if bounds_check else []
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(HERE, "..", "include", h) for h in ("evlbm.h", "evsur.h")]
    objs, jobs = [], []
    for src in sources():
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [os.path.join(CSRC, src)] + headers):
            cmd = [nvcc(), *ARCH, *COMMON, *defines, *EXTRA.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
            if ptxas_v:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or ptxas_v or r.returncode:
                print(" ".join(cmd[-3:]), r.stdout, r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    if force or jobs or not os.path.exists(lib_path):
        tmp = lib_path + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "--cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
