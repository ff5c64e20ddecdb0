"""Op-count mode of the oracle: the algorithmic work of the DARTS estimator.

TEST INFRASTRUCTURE.  Compiles darts_oracle.c a second time, as C++ with the
counting number type of opcount.hpp (every FP64 operation of the oracle's
plain restatement of the method is tallied), into oracle/liboracle_opcount.so,
and counts, per path, the forward estimator's additions, multiplications,
divisions, square roots, comparisons, exponentials, logarithms,
trigonometric functions, powers and Philox blocks.

Run as a script it writes profiles/op_counts.md: per workload of the
benchmark, the work per vertex on a fixed sample of its paths.  The
benchmark reads the roofline numerator (FP operations per vertex) from that
summary; tests/test_opcount.py recomputes it on a smaller sample and checks
the counting type itself.

    python oracle/opcount.py            # writes profiles/op_counts.md
"""
from __future__ import annotations

import ctypes as C
import fcntl
import hashlib
import json
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liboracle_opcount.so")
TALLIES = ("add", "mul", "div", "sqrt", "cmp", "exp", "log", "trig", "pow", "philox")
# FP32 operations of the algorithmic count: additions, multiplications,
# divisions (an FMA is one multiplication plus one addition); the special
# functions (square root, exp, log, trigonometric, pow) are counted apart,
# and the Philox integer work as 10 rounds x (2 wide multiplies = 4 ops,
# 4 xor, 2 key additions) = 100 integer operations per block, from the
# generator's definition (Salmon et al., SC'11).
FLOP_KINDS = ("add", "mul", "div")
SPECIAL_KINDS = ("sqrt", "exp", "log", "trig", "pow")
INT_OPS_PER_PHILOX = 100
SOURCES = ("darts_oracle.c", "darts_oracle.h", "opcount.hpp")


def source_hash() -> str:
    h = hashlib.sha256()
    for f in SOURCES:
        h.update(open(os.path.join(HERE, f), "rb").read())
    return h.hexdigest()[:16]


def build(force: bool = False) -> str:
    def stale():
        return force or not os.path.exists(LIB) or any(
            os.path.getmtime(os.path.join(HERE, f)) > os.path.getmtime(LIB) for f in SOURCES)

    if not stale():
        return LIB
    with open(os.path.join(HERE, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if stale():
            cmd = ["g++", "-O2", "-x", "c++", "-std=c++17", "-D_GNU_SOURCE", "-DORC_OPCOUNT",
                   "-include", os.path.join(HERE, "opcount.hpp"), "-fPIC", "-shared", "-pthread",
                   "-o", LIB + ".tmp", os.path.join(HERE, "darts_oracle.c"), "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        import oracle as O
        lib = C.CDLL(build())
        lib.orc_opcount_paths.argtypes = [C.POINTER(O.OrcScene), C.c_int, C.POINTER(C.c_double),
                                          C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64),
                                          C.POINTER(C.c_double)]
        lib.orc_opcount_paths.restype = C.c_int
        _lib = lib
    return _lib


def count_paths(scene, sampling, first: int, count: int, method=0, cdf=None):
    """Per-path tallies [count][10] (order of TALLIES) and vertex counts."""
    import oracle as O
    s = O.make_scene(scene, sampling)
    if method in (O.ORC_DARTS, O.ORC_DARTS_FULL_GATE) and cdf is None:
        cdf = O.build_table(scene, sampling)
    out = np.zeros((count, len(TALLIES)), np.uint64)
    nv = np.zeros(count)
    cdf_c = None if cdf is None else np.ascontiguousarray(cdf, dtype=np.float64)
    rc = load().orc_opcount_paths(C.byref(s), method, None if cdf_c is None else
                                  cdf_c.ctypes.data_as(C.POINTER(C.c_double)), first, count,
                                  out.ctypes.data_as(C.POINTER(C.c_uint64)),
                                  nv.ctypes.data_as(C.POINTER(C.c_double)))
    if rc != 0:
        raise ValueError(f"orc_opcount_paths rejected the scene ({rc})")
    return out, nv


def summarise(tallies: np.ndarray, nvert: np.ndarray) -> dict:
    tot = {k: float(tallies[:, i].sum()) for i, k in enumerate(TALLIES)}
    V = float(nvert.sum())
    n = len(nvert)
    flops = sum(tot[k] for k in FLOP_KINDS)
    special = sum(tot[k] for k in SPECIAL_KINDS)
    ints = INT_OPS_PER_PHILOX * tot["philox"]
    return {"paths": n, "vertices": V, "vertices_per_path": V / max(n, 1),
            "flops_per_vertex": flops / max(V, 1.0), "special_per_vertex": special / max(V, 1.0),
            "int_per_vertex": ints / max(V, 1.0), "cmp_per_vertex": tot["cmp"] / max(V, 1.0),
            "flops_per_path": flops / max(n, 1), "per_vertex": {k: tot[k] / max(V, 1.0) for k in TALLIES}}


def workload_sample(name: str, fraction: int = 1):
    """(scene, sampling, [(first path, count), ...], description) of the
    fixed path sample of a benchmark workload.  fraction > 1 takes every
    fraction-th piece of it (the tests' smaller sample)."""
    sys.path.insert(0, ROOT)
    from paper_2402_03106_gb300 import scenes as S
    if name == "spheres_512":
        sc = S.spheres_camera_scene(seed=0)
        sp = S.Sampling(seed=0, paths_per_element=64, max_bounces=100)
        row = 512 * 64
        pieces = [((32 + 64 * i) * row, row) for i in range(8)]  # rows 32, 96, ..., 480
        what = "rows 32 + 64 i (i < 8) of the 512x512 frame: 1/64 of its pixels, 64 spp"
    elif name == "box_camera":
        sc, sp = S.box_camera_workload(seed=0)
        pieces = [(0, 64 * 64 * 16)]
        what = "the whole 64x64 frame, 16 spp"
    elif name == "cube":
        sc, sp = S.cube_workload(paths=1 << 24, seed=0)
        pieces = [(i << 20, 1 << 14) for i in range(16)]
        what = "16 x 2^14 paths spread over the 2^24 of a step"
    else:
        raise ValueError(name)
    if fraction > 1:
        pieces = [(f, max(1, c // fraction)) for f, c in pieces]
        what += f" (1/{fraction} of each piece)"
    return sc, sp, pieces, what


def count_workload(name: str, fraction: int = 1, workers: int = 0) -> dict:
    import oracle as O
    sc, sp, pieces, what = workload_sample(name, fraction)
    cdf = O.build_table(sc, sp)
    workers = workers or min(len(pieces), os.cpu_count() or 1)
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.starmap(_count_piece, [(name, fraction, i) for i in range(len(pieces))])
    else:
        parts = [count_paths(sc, sp, f, c, O.ORC_DARTS, cdf) for f, c in pieces]
    t = np.concatenate([p[0] for p in parts])
    v = np.concatenate([p[1] for p in parts])
    out = summarise(t, v)
    out["sample"] = what
    return out


def _count_piece(name, fraction, i):
    import oracle as O
    sc, sp, pieces, _ = workload_sample(name, fraction)
    f, c = pieces[i]
    return count_paths(sc, sp, f, c, O.ORC_DARTS, O.build_table(sc, sp))


def write_summary(path: str) -> None:
    rows = {w: count_workload(w) for w in ("spheres_512", "box_camera", "cube")}
    lines = ["# Algorithmic work of the DARTS estimator (oracle op-count mode)", "",
             "command: `python oracle/opcount.py`", "",
             f"oracle_source_hash: {source_hash()}", "",
             "Counts of the oracle's own FP64 restatement of the method, compiled with a",
             "counting number type (oracle/opcount.hpp): flops = additions + multiplications",
             "+ divisions; special = square roots, exp, log, trigonometric, pow; integer =",
             "100 per Philox4x32-10 block.  Checker bookkeeping and the adjoint's score terms",
             "are not counted.  The benchmark multiplies flops_per_vertex by the vertices a",
             "launch of the path kernel reports.", "",
             "| workload | sample | paths | vertices/path | flops/vertex | special/vertex | int/vertex | cmp/vertex |",
             "|---|---|---|---|---|---|---|---|"]
    for w, r in rows.items():
        lines.append(f"| {w} | {r['sample']} | {r['paths']} | {r['vertices_per_path']:.3f} | "
                     f"{r['flops_per_vertex']:.1f} | {r['special_per_vertex']:.2f} | "
                     f"{r['int_per_vertex']:.1f} | {r['cmp_per_vertex']:.1f} |")
    lines += ["", "Per vertex, by kind:", ""]
    for w, r in rows.items():
        lines.append(f"- {w}: " + ", ".join(f"{k} {v:.2f}" for k, v in r["per_vertex"].items()))
    lines += ["", "Machine-readable (one line per workload):", ""]
    for w, r in rows.items():
        lines.append("data: " + json.dumps({"workload": w, **{k: v for k, v in r.items() if k != "per_vertex"}}))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    out = os.path.join(ROOT, "profiles", "op_counts.md")
    write_summary(out)
    print(open(out).read())
