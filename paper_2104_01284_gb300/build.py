"""Build libecodp.so in-tree with nvcc for sm_103a (GB300).

Each .cu file is compiled to an object in parallel, then linked into
paper_2104_01284_gb300/libecodp.so.  No cmake, no torch extension machinery.
build(checks=True) builds the bounds-checked variant of the same sources
(-DECODP_CHECKS) into libecodp_checked.so: every kernel index is compared
with its array's extent, failures are recorded in a device word and reported
by the host as DP_ERR_INTERNAL.  It is a debugging aid, loaded instead of the
production library when the environment variable ECODP_LIBRARY=checked.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libecodp.so")
CHECKED_LIB = os.path.join(HERE, "libecodp_checked.so")
SOURCES = ["api.cu", "api_multi.cu", "api_serve.cu", "k_precompute.cu", "k_bellman.cu", "k_rollout.cu", "k_adjoint.cu",
           "k_batch.cu", "k_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC,-O2",
         "-I" + os.path.join(os.path.dirname(HERE), "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libecodp.so")


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checks: bool = False) -> str:
    build_dir = os.path.join(BUILD, "checked") if checks else BUILD
    lib = CHECKED_LIB if checks else LIB
    flags = FLAGS + (["-DECODP_CHECKS"] if checks else [])
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "ecodp.h"))
    cc = nvcc()
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [cc, *ARCH, *flags, "-c", s, "-o", o]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out, file=sys.stderr)
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp"
        run([cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> list[str]:
    """The production library and its bounds-checked variant, compiled
    concurrently."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, force, verbose, False, c) for c in (False, True)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    if "--checks" in sys.argv:
        print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv, checks=True))
    else:
        print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
