"""Build the in-tree C-ABI library libbplg.so for sm_103a with nvcc.

Every translation unit under csrc/ is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_2310_16214_gb300/_lib/libbplg.so`` (CUDA runtime linked statically).
The benchmark's external references (extref/extref.cu: CUB, cuFFT, cuSPARSE)
go into a separate ``_lib/libbplg_extref.so`` that the library never loads.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
OBJ_DIR = os.path.join(OUT_DIR, "obj")
LIB = os.path.join(OUT_DIR, "libbplg.so")
EXTREF_SRC = os.path.join(HERE, "extref", "extref.cu")
EXTREF_LIB = os.path.join(OUT_DIR, "libbplg_extref.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(src: str, verbose_ptxas: bool) -> str:
    obj = os.path.join(OBJ_DIR, os.path.basename(src) + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj + ".tmp"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (src, r.stderr[-8000:]))
        if verbose_ptxas:
            with open(obj + ".ptxas.txt", "w") as f:
                f.write(r.stderr)
        os.replace(obj + ".tmp", obj)
    return obj


def _build_extref() -> str:
    if _stale(EXTREF_LIB, [EXTREF_SRC]):
        cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "include")
        tmp = EXTREF_LIB + ".tmp.%d" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                                 "-I" + os.path.join(cuda_inc, "cccl"), EXTREF_SRC, "-o", tmp,
                                 "-lcufft", "-lcusparse"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("extref build failed:\n" + r.stderr[-8000:])
        os.replace(tmp, EXTREF_LIB)
    return EXTREF_LIB


def build(verbose_ptxas: bool = False, jobs: int = 0) -> str:
    os.makedirs(OBJ_DIR, exist_ok=True)
    srcs = sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs + 1) as ex:
        ext = ex.submit(_build_extref)
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), srcs))
        ext.result()
    if _stale(LIB, objs):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr[-8000:])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv))
