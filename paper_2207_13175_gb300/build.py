"""Build the CUDA library ``libiod_gb300.so`` in-tree for sm_103a.

Each translation unit compiles in parallel with nvcc, then one nvcc link makes the
shared library (static CUDA runtime, so the library needs only the driver at run
time).  ``python -m paper_2207_13175_gb300.build`` rebuilds it; ``--check`` builds the
IOD_CHECK variant ``libiod_gb300_check.so`` (argument checks in the swarm kernels).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libiod_gb300.so")
BUILD_DIR = os.path.join(PKG, "_build")
# the IOD_CHECK build: the same library with the swarm kernels' argument checks compiled in
# (selected at load time by IOD_CHECK=1)
CHECK_LIB = os.path.join(PKG, "libiod_gb300_check.so")
CHECK_BUILD_DIR = os.path.join(PKG, "_build_check")
SOURCES = ["iod_kernels.cu", "iod_api.cu", "iod_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "iod.h"))
    return files


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    lib_path, build_dir = (CHECK_LIB, CHECK_BUILD_DIR) if check else (LIB, BUILD_DIR)
    if not force and not stale(lib_path):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    # host code without floating-point contraction: the few FP64 formulas the host
    # forms (the constriction factor, the line-of-sight frame) round as written
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                     "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    if check:
        common += ["-DIOD_CHECK"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def one(src: str) -> str:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [cc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, check="--check" in sys.argv))
