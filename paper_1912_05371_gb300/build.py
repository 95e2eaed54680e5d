"""Build libacm (CUDA for sm_103a + C++ host code) in-tree: paper_1912_05371_gb300/_lib/libacm.so.

Every translation unit is compiled in parallel with nvcc; no CMake.  Run as a module or call
:func:`build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libacm.so")
SOURCES = ["adjoint_f33.cu", "adjoint_d17.cu", "adjoint_f17.cu", "adjoint_d9.cu", "adjoint_f9.cu", "adapt.cu", "stage.cu", "stage_pair.cu", "api.cu",
           "topo.cu", "adjoint.cu", "forest.cpp", "noalloc.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _compile(src, obj, verbose):
    cmd = [nvcc(), "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
           "-Xcompiler", "-fopenmp",
           "--expt-relaxed-constexpr", *ARCH, "-I", os.path.join(HERE, "..", "include"), "-c",
           os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "c++")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(verbose=False, force=False):
    """Compile libacm.so if any source is newer than it; returns the library path."""
    os.makedirs(LIBDIR, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "acm.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    objs = [os.path.join(LIBDIR, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(lambda a: _compile(a[0], a[1], verbose), zip(SOURCES, objs)))
    if verbose:
        for s, l in zip(SOURCES, logs):
            sys.stderr.write(f"== {s}\n{l}")
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc(), "-shared", *ARCH, "-Xcompiler", "-fopenmp", "-o", tmp, *objs, "-lgomp"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking libacm failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
