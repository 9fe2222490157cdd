"""Build libpgm.so (the CUDA library behind include/pgm.h) in-tree for sm_103a.

    python -m paper_1911_06969_b300.build [--force] [-v] [--debug]

--debug builds libpgm_debug.so instead: the same sources with PGM_DEBUG
defined, so that the checked index sites record an out-of-range index in a
device error word (read with pgm_debug_errors) and skip the access instead
of performing it.  The package loads it when PGM_LIB=debug is set.

Every ``csrc/*.cu`` file is compiled by nvcc with
``-gencode arch=compute_103a,code=sm_103a -lineinfo`` into ``_build/`` at
the repository root and linked into ``paper_1911_06969_b300/libpgm.so``.
Objects are rebuilt when their source or any ``csrc/*.cuh`` / ``include/*.h``
header is newer.
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
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "libpgm.so")
OUT_DEBUG = os.path.join(PKG, "libpgm_debug.so")
BUILD = os.path.join(ROOT, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3,-pthread",
                     "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _newest(paths):
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    hdr_time = _newest(hdrs + [os.path.abspath(__file__)])
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    out = OUT_DEBUG if debug else OUT
    flags = NVCC_FLAGS + (["-DPGM_DEBUG"] if debug else [])
    os.makedirs(bdir, exist_ok=True)
    jobs, objs = [], []
    for s in srcs:
        o = os.path.join(bdir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_time):
            jobs.append((s, o))

    def compile_one(so):
        s, o = so
        cmd = [nvcc()] + flags + ["-c", s, "-o", o + ".tmp"]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stdout}\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for msg in ex.map(compile_one, jobs):
                if verbose and msg:
                    print(msg)
    if jobs or not os.path.exists(out) or os.path.getmtime(out) < _newest(objs):
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static", "-Xcompiler", "-pthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--debug", action="store_true", help="build libpgm_debug.so (checked index sites)")
    a = ap.parse_args(argv)
    print(build(a.force, a.verbose, a.debug))


if __name__ == "__main__":
    sys.exit(main())
