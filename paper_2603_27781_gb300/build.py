"""Builds libgs.so (the sm_103a CUDA library) in-tree with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file
and linked into paper_2603_27781_gb300/_build/libgs.so.  The CUDA runtime is
linked statically, so the library only needs the driver at run time.

With GS_CHECKS=1 in the environment (or checks=True) the checked variant is
built instead, into _build/checked/libgs.so: the blend kernels then verify the
instance ranges and items they take from the binning and report a violation
as GS_ERR_CHECK in the binning's status word (see csrc/raster.cuh).  The
binding loads the variant the environment selects.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")


def checks_requested() -> bool:
    return os.environ.get("GS_CHECKS", "0") not in ("", "0")


def lib_path(checks: bool = None) -> str:
    checks = checks_requested() if checks is None else checks
    return os.path.join(BUILD_DIR, "checked", "libgs.so") if checks else os.path.join(BUILD_DIR, "libgs.so")


LIB_PATH = lib_path()

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + SRC_DIR]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgs")


def _sources():
    return sorted(glob.glob(os.path.join(SRC_DIR, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(SRC_DIR, "*.cuh")) + [os.path.join(INCLUDE, "gs.h"), __file__]


def needs_build(checks: bool = None) -> bool:
    path = lib_path(checks)
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, checks: bool = None) -> str:
    checks = checks_requested() if checks is None else checks
    path = lib_path(checks)
    if not force and not needs_build(checks):
        return path
    nvcc = _nvcc()
    out_dir = os.path.dirname(path)
    os.makedirs(out_dir, exist_ok=True)
    flags = FLAGS + (["-DGS_CHECKS=1"] if checks else [])

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = path + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
