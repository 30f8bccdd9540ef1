"""Builds the in-tree CUDA library ``_build/libgbdct.so`` for sm_103a with nvcc.

Each ``csrc/*.cu`` translation unit is compiled in parallel (one ``-gencode``
for compute_103a / sm_103a, ``-lineinfo`` for profiling), then linked into a
shared library with a static CUDA runtime.  The build is skipped when the
library is newer than every source and header.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB_NAME = "libgbdct.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libgbdct")


def library_path() -> str:
    return os.path.join(BUILD, LIB_NAME)


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def is_stale() -> bool:
    lib = library_path()
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every CUDA source into the in-tree shared library; returns its path."""
    if not force and not is_stale():
        return library_path()
    nvcc = nvcc_path()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        logs = list(ex.map(lambda so: _compile(nvcc, so[0], so[1], extra), zip(srcs, objs)))
    if verbose or ptxas_info:
        for s, log in zip(srcs, logs):
            if log.strip():
                print(f"== {os.path.basename(s)}\n{log}")
    tmp = library_path() + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, library_path())
    return library_path()


BASELINE_LIB = "libgbdct_baselines.so"
BASELINE_SRC = os.path.join(CSRC, "baselines", "cufft_baselines.cu")


def baselines_path() -> str:
    return os.path.join(BUILD, BASELINE_LIB)


def build_baselines(force: bool = False) -> str:
    """Comparison baselines (cuFFT three-stage and row-column) in their own
    library, linked against cuFFT; the transform library does not use them."""
    out = baselines_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) > max(
            os.path.getmtime(BASELINE_SRC), os.path.getmtime(os.path.abspath(__file__))):
        return out
    os.makedirs(BUILD, exist_ok=True)
    tmp = out + ".tmp"
    cmd = [nvcc_path(), *ARCH, *NVCC_FLAGS, "-shared", BASELINE_SRC, "-o", tmp, "-lcufft", "-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"baseline build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
