"""Build libgdsw.so in-tree with nvcc for sm_103a (GB300).

Translation units compile in parallel into objects under _build/, then link into
paper_2606_01433_gb300/libgdsw.so.  Host code is portable C++17 (the same sources build on
x86_64 and aarch64).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgdsw.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["api.cu", "dense.cu", "operator.cu", "schwarz.cu", "setup.cu", "fgmres.cu", "host_setup.cpp", "noalloc.cu",
         "serve.cpp", "probe.cu", "tc_gemm.cu", "mg.cu"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _compile(unit: str, verbose: bool) -> str:
    src = os.path.join(SRC, unit)
    obj = os.path.join(BUILD, unit + ".o")
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
           "-Xcompiler", "-fPIC,-O3", "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    if unit.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, r.stdout, r.stderr))
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    for f in os.listdir(SRC):
        if os.path.getmtime(os.path.join(SRC, f)) > t:
            return True
    if os.path.getmtime(os.path.join(ROOT, "include", "gdsw.h")) > t:
        return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, len(UNITS))) as ex:
        objs = list(ex.map(lambda u: _compile(u, verbose), UNITS))
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", OUT + ".tmp", *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
