"""Build libmcubes.so in-tree for sm_103a with nvcc.

Every translation unit under csrc/ is compiled in parallel. The V-Sample instances are one
unit per (precision, integrand) slice. The objects are linked into
paper_2302_05730_gb300/libmcubes.so with the CUDA runtime linked statically, so loading the
library needs only the driver. Objects are rebuilt when a source or header is newer.

    python -m paper_2302_05730_gb300.build [--force] [--jobs N] [--checked]

--checked builds a separate library, libmcubes_checked.so (objects in _build_checked), whose
kernels check every computed bin, sub-cube and probe index against its bound and count failures
(mcubes_checked_violations) instead of accessing out of bounds. Load it with MCUBES_LIB.

MCUBES_NVCC_EXTRA adds nvcc flags to every unit (objects are not rebuilt when only it changes:
use --force).
"""
from __future__ import annotations

import argparse
import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libmcubes.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libmcubes_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _units():
    """(object name, source, extra defines) for every translation unit."""
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        name = os.path.splitext(os.path.basename(src))[0]
        if name == "vsample_inst":
            for f32 in (0, 1):
                for fid in range(10):
                    for part in (0, 1):   # 0: single-job kernels, 1: batched kernels
                        units.append((f"vsample_{'f32' if f32 else 'f64'}_{fid}_{'batch' if part else 'one'}", src,
                                      [f"-DMCUBES_F32={f32}", f"-DMCUBES_FID={fid}", f"-DMCUBES_PART={part}"]))
        else:
            units.append((name, src, []))
    return units


def _deps_mtime():
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hdrs) if hdrs else 0.0


def build(force: bool = False, jobs: int | None = None, checked: bool = False, verbose: bool = False) -> str:
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    dep_t = _deps_mtime()
    extra = ["-DMCUBES_CHECKED=1"] if checked else []
    extra += os.environ.get("MCUBES_NVCC_EXTRA", "").split()   # extra nvcc flags (e.g. -D overrides)
    todo, objs = [], []
    for name, src, defs in _units():
        obj = os.path.join(build_dir, name + ".o")
        objs.append(obj)
        stale = force or not os.path.exists(obj) or \
            os.path.getmtime(obj) < max(os.path.getmtime(src), dep_t)
        if stale:
            todo.append([nvcc] + NVCC_FLAGS + extra + defs + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with ThreadPoolExecutor(max_workers=n) as ex:
            list(ex.map(run, todo))
    if todo or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        run([nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs)
        os.replace(tmp, lib)
    return lib


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--checked", action="store_true", help="bounds-checked kernels")
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, jobs=a.jobs, checked=a.checked, verbose=a.verbose))


if __name__ == "__main__":
    main()
