"""Build libdarts.so in-tree with nvcc for sm_103a (no GPU needed to compile).

Each translation unit under csrc/ is compiled in parallel into
paper_2402_03106_gb300/_build/, then linked into
paper_2402_03106_gb300/libdarts.so next to this file.  The checked variant
(libdarts_checked.so, objects in _build_checked/) is built beside it.
"""
from __future__ import annotations

import fcntl
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdarts.so")
SOURCES = ["capi.cu", "table.cu", "trace.cu", "trace_var.cu"]
HEADERS = ["darts_device.cuh", "darts_internal.h", "trace_kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The path kernels take FP32 division and square root at 2 ulp / 1 ulp
# (div.full, sqrt.approx) instead of IEEE rounding: shorter dependent chains,
# well inside the per-path FP32 error budget.  The table build keeps IEEE.
APPROX_SOURCES = {"trace.cu", "trace_var.cu"}
APPROX_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose: bool) -> list:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


# Variants: (library, object directory, extra nvcc flags).  The checked
# library tests every output, tile and table index on the device
# (-DDARTS_CHECKS); it shares all sources with the production one.
CHECKED_LIB = os.path.join(HERE, "libdarts_checked.so")
VARIANTS = [(LIB, BUILD, []), (CHECKED_LIB, os.path.join(HERE, "_build_checked"), ["-DDARTS_CHECKS"])]


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [
        os.path.join(ROOT, "include", "darts.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Build libdarts.so (and libdarts_checked.so) when a source is newer;
    returns the production library's path."""
    variants = VARIANTS if checked else VARIANTS[:1]
    if not force and not any(_stale(lib) for lib, _, _ in variants):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # one builder at a time (ranks of a multi-process launch build together)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        todo = [v for v in variants if force or _stale(v[0])]
        if todo:
            _build_locked(todo, verbose)
    return LIB


def _build_locked(variants, verbose: bool) -> None:
    cc = nvcc()
    flags = _flags(verbose)

    def compile_one(job) -> str:
        src, out_dir, defs = job
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        extra = APPROX_FLAGS if src in APPROX_SOURCES else []
        cmd = [cc] + flags + extra + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {' '.join(defs)}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    jobs = []
    for _, out_dir, defs in variants:
        os.makedirs(out_dir, exist_ok=True)
        jobs += [(src, out_dir, defs) for src in SOURCES]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (lib, _, _) in enumerate(variants):
        tmp = lib + ".tmp"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs[k * len(SOURCES):(k + 1) * len(SOURCES)] + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
