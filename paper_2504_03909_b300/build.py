"""Builds the native library ``libpaillier_b300.so`` in-tree with nvcc for sm_103a.

    python -m paper_2504_03909_b300.build [--jobs N] [--force] [--checked]

Each translation unit under ``csrc/`` is compiled to ``_build/*.o`` (in
parallel; an object is rebuilt when its source or any header is newer), then
linked into ``paper_2504_03909_b300/libpaillier_b300.so`` with the CUDA
runtime linked statically, so the library carries no dependency on a
particular libcudart on the loading side.  ``--checked`` builds the same
sources with device-side bounds checks (-DPL_CHECKED, see csrc/check.cuh) into
``libpaillier_b300_checked.so`` (objects in ``_build_checked/``).
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpaillier_b300.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libpaillier_b300_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(src: str, checked: bool = False):
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(PKG, "..", "include")]
    if checked:
        common.append("-DPL_CHECKED")
    if src.endswith(".cu"):
        return ARCH + common + ["-lineinfo", "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
    return common + ["-x", "cu"] + ARCH  # host C++ files still go through nvcc (CUDA runtime headers)


def _newest_header() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    hs += glob.glob(os.path.join(PKG, "..", "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, force: bool, verbose: bool, checked: bool = False) -> str:
    obj = os.path.join(BUILD_CHECKED if checked else BUILD, os.path.basename(src) + ".o")
    if not force and os.path.exists(obj):
        t = os.path.getmtime(obj)
        if t >= os.path.getmtime(src) and t >= _newest_header():
            return obj
    cmd = [nvcc()] + _flags(src, checked) + ["-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip() and verbose:
        print(r.stderr, file=sys.stderr)
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, checked: bool = False) -> str:
    bdir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, verbose, checked), srcs))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", lib] + objs + ["-lpthread"]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--checked", action="store_true", help="build the bounds-checked library")
    a = ap.parse_args()
    print(build(force=a.force, jobs=a.jobs, verbose=a.verbose, checked=a.checked))


if __name__ == "__main__":
    main()
