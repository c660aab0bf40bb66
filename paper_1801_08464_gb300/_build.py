"""Compile the CUDA library (sm_103a) in-tree: paper_1801_08464_gb300/_lib/libmgrgpu.so.

One nvcc process per translation unit, run in parallel, then a shared link.  The setup units
(sparse.cu, setup.cu) are built with --fmad=false: their arithmetic is a fixed sequence of IEEE
operations.  The apply / Krylov units use the default contraction.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIBPATH = os.path.join(LIBDIR, "libmgrgpu.so")
OBJDIR = os.path.join(LIBDIR, "obj")
UNITS = ["scan.cu", "sparse.cu", "setup.cu", "sell.cu", "rowsop.cu", "apply.cu", "krylov.cu", "mgr.cu", "noalloc.cu", "probe.cu"]
NOFMA = {"sparse.cu", "setup.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "mgr.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIBPATH) and os.path.getmtime(LIBPATH) >= _sources_mtime():
        return LIBPATH
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                     "--expt-relaxed-constexpr"]

    def compile_unit(u: str) -> str:
        obj = os.path.join(OBJDIR, u.replace(".cu", ".o"))
        cmd = [nvcc, *common, "-c", os.path.join(CSRC, u), "-o", obj]
        if u in NOFMA:
            cmd.insert(1, "--fmad=false")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIBPATH + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIBPATH)
    return LIBPATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))
