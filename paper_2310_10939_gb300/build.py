"""Build libfsc.so in-tree: one nvcc per translation unit (in parallel), then a shared link.

Usage: python -m paper_2310_10939_gb300.build [--force] [--verbose] [--bounds-check]
Targets sm_103a only (GB300).  Objects go to ``_build/`` next to this file.  --bounds-check
builds libfsc_checked.so (objects in ``_build_checked/``) with -DFSC_BOUNDS_CHECK: every
input-derived index is tested before its access and the first violation is recorded
(fsc_bounds_report); the binding loads it when FSC_LIBRARY=checked.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfsc.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libfsc_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-O3"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfsc.so")
    return path


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None, bounds_check: bool = False) -> str:
    build_dir, lib_path = (BUILD_CHECKED, LIB_CHECKED) if bounds_check else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "fsc.h"))
    extra = list(extra_flags or []) + (["-DFSC_BOUNDS_CHECK"] if bounds_check else [])
    jobs = []
    for src in sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src[:-3] + ".o")
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *FLAGS, *extra, "-c", s, "-o", o])
    objs = [os.path.join(build_dir, src[:-3] + ".o") for src in sources()]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    failed = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or r.returncode:
                    sys.stderr.write(" ".join(cmd[-3:]) + "\n" + r.stdout + r.stderr)
                if r.returncode:
                    failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    if force or jobs or _stale(lib_path, objs):
        cmd = [nvcc(), *ARCH, "-shared", "-o", lib_path, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    return lib_path


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true", help="print register/smem usage per kernel")
    ap.add_argument("--bounds-check", action="store_true", help="build libfsc_checked.so with -DFSC_BOUNDS_CHECK")
    args = ap.parse_args()
    extra = ["-Xptxas", "-v"] if args.ptxas_v else []
    print(build(force=args.force or args.ptxas_v, verbose=args.verbose or args.ptxas_v, extra_flags=extra,
                bounds_check=args.bounds_check))
