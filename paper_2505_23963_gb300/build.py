"""Compile the CUDA library in-tree: ``paper_2505_23963_gb300/_lib/libfdtdbath.so``.

Every translation unit is compiled by nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a -lineinfo``), in parallel, and linked
into one shared library with a static CUDA runtime.  The FP64 kernels and the
FP64 reductions are compiled with ``--fmad=false`` so that each multiply and add
rounds on its own, the order in which the equations are written; the bath
recursion's explicit fused multiply-adds (the same in every kernel) are the
exception.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libfdtdbath.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]
# (source, extra flags)
UNITS = [
    ("api.cpp", []),
    ("step3d_f32.cu", []),
    ("step3d_f64.cu", ["--fmad=false"]),
    ("plain3d_f32.cu", []),
    ("plain3d_sig_f32.cu", []),
    ("plain3d_f64.cu", ["--fmad=false"]),
    ("te2d_f32.cu", []),
    ("tb2_f32.cu", []),
    ("tb2_f64.cu", ["--fmad=false"]),
    ("reduce.cu", ["--fmad=false"]),
    ("noalloc.cu", ["--fmad=false"]),
    ("peak.cu", []),
    ("cavity1d_f32.cu", []),
    ("cavity1d_f64.cu", ["--fmad=false"]),
    ("batch.cpp", []),
    ("batch1d_f32.cu", []),
    ("batch1d_f64.cu", ["--fmad=false"]),
    ("adjoint_f32.cu", []),
    ("adjoint_f64.cu", ["--fmad=false"]),
]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the library if any source is newer than it; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources_mtime():
        return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(unit):
        src, extra = unit
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + COMMON + extra
        if src.endswith(".cpp"):
            cmd += ["-x", "cu"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
        if verbose and res.stderr:
            print(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(UNITS))) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + ARCH + objs + ["-cudart=static"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
