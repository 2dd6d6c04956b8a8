"""Build the CUDA library in-tree: paper_2508_11790_gb300/_lib/libbs_mvdr.so.

Each translation unit is compiled in parallel (nvcc for .cu with one
-gencode for sm_103a, g++ for the host .cpp files with -ffp-contract=off),
then linked into one shared library with the CUDA runtime linked statically.
Usage: python -m paper_2508_11790_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
BUILD_DIR = os.path.join(ROOT, "_build", "bs_mvdr")
LIB_NAME = "libbs_mvdr.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def lib_path() -> str:
    return os.path.join(OUT_DIR, LIB_NAME)


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                 + glob.glob(os.path.join(INCLUDE, "*.h")))
    return cu, cpp, hdr


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    if verbose and r.stdout.strip():
        print(r.stdout)
    return r.stdout


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    cu, cpp, hdr = _sources()
    out = lib_path()
    if not force and not _stale(out, cu + cpp + hdr + [__file__]):
        return out
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    incs = ["-I" + INCLUDE, "-I" + CSRC, "-I" + os.path.join(home, "include")]
    jobs = []
    for src in cu:
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "--expt-relaxed-constexpr", "-c", src, "-o", obj] + incs
        if ptxas_verbose:
            cmd.append("-Xptxas=-v")
        jobs.append((obj, cmd))
    for src in cpp:
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-c", src, "-o", obj] + incs
        jobs.append((obj, cmd))
    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(_run, cmd, verbose) for _, cmd in jobs]
        for f in futs:
            logs.append(f.result())
    tmp = out + ".tmp"
    _run([nvcc, ARCH, "-shared", "-cudart=static", "-o", tmp] + [o for o, _ in jobs]
         + ["-Xlinker", "-soname=" + LIB_NAME], verbose)
    os.replace(tmp, out)
    if ptxas_verbose:
        print("\n".join(l for l in logs if l.strip()))
    return out


if __name__ == "__main__":
    path = build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                 ptxas_verbose="--ptxas" in sys.argv)
    print(path)
