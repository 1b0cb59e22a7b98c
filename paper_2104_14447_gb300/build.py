"""Build libgmls.so (sm_103a) in-tree with nvcc.

``python -m paper_2104_14447_gb300.build`` or ``build()``; translation units
compile in parallel, then link into ``_build/libgmls.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgmls.so")
SOURCES = ["capi.cu", "nbr.cu", "stencil.cu", "stencil_fast.cu", "noalloc.cu", "serve.cu", "stokes.cu", "krylov.cu", "fast_s2a.cu",
           "fast_s2b.cu", "fast_s2c.cu", "fast_s3a.cu", "fast_s3b.cu", "fast_s3c.cu", "fast_d2.cu", "fast_d3.cu", "fast_g2.cu", "fast_g3.cu", "fast_n.cu", "fast_s2d.cu", "dfx.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: libgmls needs the CUDA toolkit")
    return exe


def _inputs_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(HERE, "..", "include", "gmls.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths if os.path.isfile(p))


def _gen_tables() -> None:
    hdr = os.path.join(CSRC, "basis_tables.cuh")
    gen = os.path.join(CSRC, "basisgen.py")
    if not os.path.exists(hdr) or os.path.getmtime(hdr) < os.path.getmtime(gen):
        subprocess.run([sys.executable, gen], check=True, cwd=CSRC, stdout=subprocess.DEVNULL)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile every CUDA translation unit for sm_103a and link libgmls.so."""
    _gen_tables()
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _inputs_mtime():
        return LIB
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(HERE, "..", "include")]
    flags += list(extra_flags or [])
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [exe, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([exe, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
