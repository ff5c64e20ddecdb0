#!/usr/bin/env python3
"""Throughput benchmark of the DARTS hot path on GB300.

One step = one pass of the whole path over one frame of the workload: the
elliptical DA direction table is rebuilt on the GPU (the same launch zeroes
the frame's histograms), then every path of the frame is traced (DA-RIS
distance sampling, EDA/MIS directions, elliptical control vertices, surface
bounces) and accumulated into per-pixel time-bin histograms.

Default workload (``--workload spheres_512``), the largest configuration that
fits one GPU: a 512x512 pinhole camera (40 deg FOV) inside a 4x4x4 medium
(sigma_s 0.8, sigma_a 0.005, g 0.8) holding 32 seeded Lambertian spheres,
lit by two point pulse emitters (t0 = 0 and 1.5); 1000 bins on [0, 20);
64 paths per pixel (16.7 M per frame), 100 bounces, 8 RIS candidates,
16x8x256 direction table; a 2.1 GB FP64 histogram per frame.
``--workload box_camera`` is the 64x64 walled box with the area emitter
(512 bins, 16 spp); ``--workload cube`` the unit-cube medium with point
emitter and sensor at 2^24 paths per step.  The default run also reports
those two, compactly.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
  python bench.py --studies OUT.json     # efficiency and side studies, to a file
  python bench.py --only {timed,batched,differentiable}

stdout carries exactly one line: the JSON headline.  The efficiency
comparisons (MSE x time against the uniform-temporal and vanilla tracers,
ablations, gates), the batched launch, the differentiable step and frames
in flight run only with ``--studies`` and are written to that file.

Under torchrun every rank traces its own path-id range (weak scaling) and the
per-rank histograms are combined with one FP64 all-reduce per step, which
runs while the next step renders (two histogram buffers alternate).  The
``--impl reference`` arm times the FP64 CPU oracle on this host's cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DARTS transient path samples/s on 1 GB300; MSE×time vs plain transient PT"
WORKLOADS = {
    "spheres_512": ("512x512 pinhole camera (FOV 40 deg) at (2,2,0.05) looking +z inside a 4x4x4 medium "
                    "sigma_s 0.8 sigma_a 0.005 g 0.8; 32 seeded Lambertian spheres (r U[0.05,0.3], albedo "
                    "U[0.2,0.8]); two point pulse emitters (1,3.5,1) t0=0 and (3,3.5,3) t0=1.5; 1000 bins on "
                    "[0,20); 64 spp (16.7 M paths per frame), K=100, N_RIS=8, table 16x8x256; 2.1 GB FP64 "
                    "histogram; one frame per GPU per step"),
    "spheres_256": ("the spheres_512 scene seen at 256x256 (4.2 M paths, a 0.52 GB histogram): the small "
                    "case of the same kernel for profiler captures"),
    "box_camera": ("64x64 pinhole camera (FOV 40 deg) at (1,1,-2.5) viewing a 2x2x2 box, five Lambertian "
                   "walls albedo 0.5 (front face open); medium from seed 0: sigma_s U[0.5,2], albedo "
                   "U[0.9,0.99], g U[0,0.9]; 0.3x0.3 Lambertian area pulse emitter on the ceiling, t0=0; "
                   "512 bins on [0,16); 16 spp (65536 paths per frame), K=50, N_RIS=8, table 16x8x256"),
    "cube": ("unit-cube medium sigma_s=1 sigma_a=0.01 g=0.7 v=1; isotropic point pulse emitter "
             "(0.5,0.5,0.1) t0=0; point fluence sensor (0.5,0.5,0.9); 256 bins on [0.8,6.0); "
             "K=50 bounces, N_RIS=8, table 16x8x256; 2^24 paths per GPU per step"),
}
DEFAULT_STEPS = {"spheres_512": 30, "spheres_256": 60, "box_camera": 2000, "cube": 60}
SM_COUNT = 152
FP32_LANES_PER_SM = 128
MUFU_PER_SM_CLK = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 30 frames of the 512x512 workload, 2000 box frames, 60 cube steps)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="spheres_512", choices=sorted(WORKLOADS))
    ap.add_argument("--studies", default=None, metavar="OUT.json",
                    help="also run the efficiency and side studies and write them to this file")
    ap.add_argument("--only", default=None, choices=["timed", "batched", "differentiable"],
                    help="run one measurement alone (for ncu captures of its kernels)")
    ap.add_argument("--only-timed", action="store_true", help="same as --only timed")
    ap.add_argument("--launch", default=None, metavar="BLOCK,CHUNK",
                    help="path-kernel launch shape instead of the autotuner's (profiler captures: "
                         "no tuning launches before the timed ones)")
    a = ap.parse_args()
    if a.only_timed:
        a.only = "timed"
    if a.steps is None:
        a.steps = DEFAULT_STEPS[a.workload]
    return a


def make_workload(name, S):
    """(scene, sampling, paths per step) of a named workload."""
    if name in ("spheres_512", "spheres_256"):
        side = 512 if name == "spheres_512" else 256
        sc = S.spheres_camera_scene(seed=0, width=side, height=side)
        sp = S.Sampling(seed=0, paths_per_element=64, max_bounces=100)
    elif name == "box_camera":
        sc, sp = S.box_camera_workload(seed=0)
    else:
        sc, sp = S.cube_workload(paths=1 << 24, seed=0)
    sp.flags |= S.FLAG_REBUILD_TABLE
    return sc, sp, S.total_paths(sc, sp)


def oracle_sample(name, S):
    """The bounded oracle sample of a workload: a list of (first path id,
    path count, (first element, element count)) pieces and its description.
    512x512 frame: rows 32 + 64 i (i < 8), 1/64 of the pixels at 64 spp."""
    sc, sp, n = make_workload(name, S)
    if name == "spheres_512":
        row = 512 * 64
        pieces = [((32 + 64 * i) * row, row, ((32 + 64 * i) * 512, 512)) for i in range(8)]
        return pieces, "rows 32 + 64 i (i < 8) of the 512x512 frame: 1/64 of its pixels, 64 spp each"
    if name == "spheres_256":
        row = 256 * 64
        pieces = [((16 + 32 * i) * row, row, ((16 + 32 * i) * 256, 256)) for i in range(8)]
        return pieces, "rows 16 + 32 i (i < 8) of the 256x256 frame: 1/32 of its pixels, 64 spp each"
    if name == "box_camera":
        return [(0, n, None)], "one whole 64x64 frame (65536 paths)"
    return [(0, 1 << 22, None)], "2^22 paths of the 2^24-path step"


# ----------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("trace_kernels.cuh", "trace.cu", "darts_device.cuh", "darts_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2402_03106_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, paths_per_launch: int):
    """DRAM bytes per launch of the trace kernel from the committed ncu
    summary of this workload, when it was taken on the current source; a
    capture of a smaller launch is scaled by the paths when the summary says
    its traffic grows with them."""
    path = os.path.join(ROOT, "profiles", f"darts_trace_kernel_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+-]+)", text)
    m_paths = re.search(r"paths_per_launch:\s*([0-9]+)", text)
    m_scale = re.search(r"traffic_scales_with_paths:\s*(yes|no)", text)
    if not (m_hash and m_bytes and m_paths) or m_hash.group(1) != kernel_source_hash():
        return None
    v = float(m_bytes.group(1))
    if m_scale and m_scale.group(1) == "yes":
        v *= paths_per_launch / float(m_paths.group(1))
    return v


def algorithmic_work(workload: str):
    """Work per vertex of a workload from the oracle's op-count summary
    (profiles/op_counts.md, written by oracle/opcount.py): FP operations
    (add, mul, div), special functions (sqrt, exp, log, trig, pow) and
    Philox integer operations."""
    try:
        text = open(os.path.join(ROOT, "profiles", "op_counts.md")).read()
    except OSError:
        return None
    for line in text.splitlines():
        if line.startswith("data: "):
            d = json.loads(line[len("data: "):])
            if d.get("workload") == workload:
                return d
    return None


# ----------------------------------------------------------------------------
def cpu_baseline(workload: str, budget_s: float = 10.0):
    """The FP64 oracle, as it stands, on this host's cores: the bounded
    sample of the workload (for the 512x512 frame, 1/64 of its pixels),
    repeated over successive frames until about budget_s has passed;
    paths/s of the sample extrapolate to the whole frame by path count."""
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    sc, sp, N = make_workload(workload, S)
    pieces, what = oracle_sample(workload, S)
    cores = os.cpu_count() or 1
    cdf = O.build_table(sc, sp)
    done, paths, t_tot = 0, 0, 0.0
    while t_tot < budget_s and done < 128:
        for first, count, window in pieces:
            t0 = time.perf_counter()
            O.render(sc, sp, O.ORC_DARTS, n_paths=count, offset=first + done * N, cdf=cdf, threads=cores,
                     window=window)
            t_tot += time.perf_counter() - t0
            paths += count
        done += 1
    first, count, window = pieces[0]
    n1 = max(1, count // 2)
    t0 = time.perf_counter()
    O.render(sc, sp, O.ORC_DARTS, n_paths=n1, offset=first, cdf=cdf, threads=1, window=window)
    t1 = time.perf_counter() - t0
    return {"value": paths / t_tot, "unit": "paths/s", "cores": cores, "kind": "oracle",
            "sample": f"{what}; {done} frame(s) of that sample ({paths} paths, direction table prebuilt), "
                      f"FP64 C oracle, {cores} POSIX threads, {t_tot:.2f} s wall; paths/s of the sample "
                      f"(a whole frame extrapolates by its path count)",
            "single_thread": {"value": n1 / t1, "unit": "paths/s", "cores": 1,
                              "sample": f"{n1} paths of the same sample, {t1:.2f} s wall"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    cores = os.cpu_count() or 1
    sc, sp, N = make_workload(args.workload, S)
    pieces, what = oracle_sample(args.workload, S)
    # the FP64 table build (about 0.1 s) is done once, before the timed steps,
    # so that any step count stays within minutes
    cdf = O.build_table(sc, sp)
    times, paths = [], 0
    for i in range(args.warmup + args.steps):
        first, count, window = pieces[i % len(pieces)]
        t0 = time.perf_counter()
        O.render(sc, sp, O.ORC_DARTS, n_paths=count, offset=first + (i // len(pieces)) * N, cdf=cdf,
                 threads=cores, window=window)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            paths += count
    tot = sum(times)
    value = paths / tot
    step_what = (f"one piece of the sample per step ({pieces[0][1]} paths), cycling over: {what}; "
                 f"direction table built once before the timed steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "paths/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                       "reference_sample": step_what},
            "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cores, "kind": "oracle",
                             "sample": f"{step_what}, {cores} POSIX threads"},
            "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
def mse_time(ctx, S, torch, n_paths=1 << 20, seeds=16):
    """Efficiency of DARTS against the plain uniform-temporal path tracer (and
    the vanilla direct-connection tracer, the ablations of Fig. 13 and the
    RIS variants of Sec. 4.3) at
    equal path counts, on the benchmark's unit cube and on a paper-shaped dense
    variant (sigma_s = 13.5: about 3.2 transport mean free paths between
    emitter and sensor).

    With a point emitter every estimator here has infinite variance (the
    control vertex next to the emitter), so two figures are reported per
    method: the MSE against the pooled mean of all renders (mean and median
    over seeds), and a robust spread -- the interquartile range over seeds of
    each bin.  ratio_* = (spread^2 x time)_base / (spread^2 x time)_darts,
    median over bins; render time (table build + trace) from CUDA events."""
    methods = (("darts", S.DARTS, 0), ("darts_no_da", S.DARTS, S.FLAG_NO_DA_DISTANCE),
               ("darts_no_eda", S.DARTS, S.FLAG_NO_EDA),
               ("darts_no_da_no_eda", S.DARTS, S.FLAG_NO_DA_DISTANCE | S.FLAG_NO_EDA),
               ("darts_iid_candidates", S.DARTS, S.FLAG_IID_CANDIDATES),
               ("darts_equiangular", S.DARTS, S.FLAG_EQUIANGULAR),
               ("darts_reservoir", S.DARTS, S.FLAG_RESERVOIR),
               ("plain_uniform_t", S.PLAIN_UNIFORM_T, 0), ("vanilla_direct", S.VANILLA_DIRECT, 0))
    out = {"paths_per_render": n_paths, "seeds": seeds}
    for label, sc in (("unit_cube", S.slab_scene()), ("unit_cube_sigma_s_13.5", S.slab_scene(sigma_s=13.5))):
        H, T = {}, {}
        for name, m, fl in methods:
            hs, ts = [], []
            for s_ in range(seeds):
                sp = S.Sampling(seed=7 + s_, paths_per_element=n_paths, method=m,
                                flags=fl | (S.FLAG_REBUILD_TABLE if m == S.DARTS else 0))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                h = ctx.render(sc, sp)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e-3)
                hs.append(h)
            H[name] = torch.stack(hs).cpu()
            T[name] = statistics.median(ts)
        ref = torch.cat([H[n] for n, m, _ in methods if m != S.VANILLA_DIRECT]).mean(0)
        res = {}
        for name, _, _ in methods:
            d = H[name] - ref
            mse = (d * d).mean(1)
            q = torch.quantile(H[name], torch.tensor([0.25, 0.75], dtype=torch.float64), dim=0)
            res[name] = {"seconds_per_render": T[name], "mse_mean": float(mse.mean()),
                         "mse_median": float(mse.median()), "_iqr": (q[1] - q[0])}
        for base in ("plain_uniform_t", "vanilla_direct", "darts_no_da", "darts_no_eda", "darts_no_da_no_eda",
                     "darts_iid_candidates", "darts_equiangular", "darts_reservoir"):
            a = res[base]["_iqr"] ** 2 * res[base]["seconds_per_render"]
            b = res["darts"]["_iqr"] ** 2 * res["darts"]["seconds_per_render"]
            ok = (a > 0) & (b > 0)
            res[f"ratio_{base}_over_darts"] = {
                "robust_spread2_time_median_over_bins": float((a[ok] / b[ok]).median()) if ok.any() else None,
                "mse_mean_time": (res[base]["mse_mean"] * res[base]["seconds_per_render"]) /
                                 max(res["darts"]["mse_mean"] * res["darts"]["seconds_per_render"], 1e-300),
                "mse_median_time": (res[base]["mse_median"] * res[base]["seconds_per_render"]) /
                                   max(res["darts"]["mse_median"] * res["darts"]["seconds_per_render"], 1e-300)}
        for name in res:
            if isinstance(res[name], dict):
                res[name].pop("_iqr", None)
        out[label] = res
    return out


def mse_time_camera(ctx, S, torch, seeds=16, spps=(16, 64)):
    """Config-2 comparison: the walled box seen by the 64x64 camera (512 bins),
    DARTS against the plain uniform-temporal tracer and the vanilla
    direct-connection tracer, 16 seeds per method and sample count.  MSE per
    render against the pooled mean of every DARTS and plain render (all
    pixels and bins); ratio = (MSE x time)_base / (MSE x time)_darts with the
    median render time (table build + trace, CUDA events)."""
    sc = S.box_camera_scene(seed=0)
    methods = (("darts", S.DARTS), ("plain_uniform_t", S.PLAIN_UNIFORM_T), ("vanilla_direct", S.VANILLA_DIRECT),
               ("darts_full_gate", S.DARTS_FULL_GATE))
    out = {"workload": "box camera of the benchmark, 64x64, 512 bins, K=50", "seeds": seeds}
    for spp in spps:
        H, T = {}, {}
        for name, m in methods:
            acc, ts = [], []
            for s_ in range(seeds):
                sp = S.Sampling(seed=101 + s_, paths_per_element=spp, max_bounces=50, method=m,
                                flags=S.FLAG_REBUILD_TABLE if m in (S.DARTS, S.DARTS_FULL_GATE) else 0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                h = ctx.render(sc, sp)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e-3)
                acc.append(h.reshape(-1).float())
            H[name] = torch.stack(acc)
            T[name] = statistics.median(ts)
        ref = torch.cat([H["darts"], H["plain_uniform_t"]]).double().mean(0).float()
        res = {}
        for name, _ in methods:
            d = H[name] - ref
            mse = (d * d).double().mean(1)
            res[name] = {"seconds_per_render": T[name], "mse_mean": float(mse.mean()),
                         "mse_median": float(mse.median())}
        for base in ("plain_uniform_t", "vanilla_direct", "darts_full_gate"):
            res[f"ratio_{base}_over_darts"] = {
                "mse_mean_time": (res[base]["mse_mean"] * res[base]["seconds_per_render"]) /
                                 max(res["darts"]["mse_mean"] * res["darts"]["seconds_per_render"], 1e-300),
                "mse_median_time": (res[base]["mse_median"] * res[base]["seconds_per_render"]) /
                                   max(res["darts"]["mse_median"] * res["darts"]["seconds_per_render"], 1e-300)}
        res["ratio_plain_uniform_t_over_darts_full_gate"] = {
            "mse_mean_time": (res["plain_uniform_t"]["mse_mean"] * res["plain_uniform_t"]["seconds_per_render"]) /
                             max(res["darts_full_gate"]["mse_mean"] * res["darts_full_gate"]["seconds_per_render"], 1e-300)}
        out[f"spp_{spp}"] = res
        del H
    return out


def mse_time_gated(ctx, S, torch, seeds=16, spp=64):
    """Time-gated rendering (one gate, one bin), the regime of the paper's
    time-gated experiments: the walled box seen by the 64x64 camera, gates of
    width w centred at t, DARTS against the uniform-temporal and vanilla
    tracers.  MSE per render against the pooled mean of the DARTS and
    uniform-temporal renders; ratio = (MSE x time)_base / (MSE x time)_darts."""
    out = {"workload": "box camera of the benchmark, 64x64, one gate bin, K=100", "seeds": seeds, "spp": spp}
    methods = (("darts", S.DARTS), ("plain_uniform_t", S.PLAIN_UNIFORM_T), ("vanilla_direct", S.VANILLA_DIRECT))
    cases = [(6.125, 0.25, spp), (10.125, 0.25, spp), (8.0, 0.0625, spp), (8.0, 1.0, spp), (8.0, 4.0, spp),
             (6.125, 0.25, 1024), (10.125, 0.25, 1024)]  # the last two GPU-saturating (4 M paths)
    for centre, width, spp_c in cases:
        sc = S.box_camera_scene(seed=0, n_bins=1, t_max=centre + width / 2)
        sc.gate.t_min = centre - width / 2
        H, T = {}, {}
        for name, m in methods:
            acc, ts = [], []
            for s_ in range(seeds):
                sp = S.Sampling(seed=301 + s_, paths_per_element=spp_c, max_bounces=100, method=m,
                                flags=S.FLAG_REBUILD_TABLE if m == S.DARTS else 0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                h = ctx.render(sc, sp)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e-3)
                acc.append(h.reshape(-1))
            H[name] = torch.stack(acc)
            T[name] = statistics.median(ts)
        ref = torch.cat([H["darts"], H["plain_uniform_t"]]).mean(0)
        res = {"gate": [centre - width / 2, centre + width / 2], "spp": spp_c, "mean_signal": float(ref.mean())}
        for name, _ in methods:
            d = H[name] - ref
            mse = (d * d).mean(1)
            res[name] = {"seconds_per_render": T[name], "mse_mean": float(mse.mean()),
                         "mse_median": float(mse.median())}
        for base in ("plain_uniform_t", "vanilla_direct"):
            res[f"ratio_{base}_over_darts"] = {
                "mse_mean_time": (res[base]["mse_mean"] * res[base]["seconds_per_render"]) /
                                 max(res["darts"]["mse_mean"] * res["darts"]["seconds_per_render"], 1e-300),
                "mse_median_time": (res[base]["mse_median"] * res[base]["seconds_per_render"]) /
                                   max(res["darts"]["mse_median"] * res["darts"]["seconds_per_render"], 1e-300)}
        out[f"gate_{centre - width / 2:g}_{centre + width / 2:g}_spp{spp_c}"] = res
    return out


def mse_time_gated_dense(ctx, S, torch, seeds=24, paths=1 << 18):
    """Time-gated rendering deep in a dense medium, the regime the diffusion
    approximation describes: an infinite medium (sigma_s = 10, sigma_a =
    0.01), point emitter and fluence sensor 3 transport mean free paths
    apart, one gate bin.  Isotropic scattering (separation 0.3) and g = 0.7
    (separation 1.0).  Per method: `seeds` renders of `paths` paths; the
    single-bin estimates have heavy tails (point emitter), so the spread is
    reported as the interquartile range beside the MSE against the median of
    the pooled DARTS and uniform-temporal estimates.  efficiency = 1 /
    (spread^2 x time); ratio = efficiency of DARTS / efficiency of the
    method."""
    import numpy as np
    methods = (("darts", S.DARTS, 0), ("darts_no_da", S.DARTS, S.FLAG_NO_DA_DISTANCE),
               ("darts_no_eda", S.DARTS, S.FLAG_NO_EDA), ("plain_uniform_t", S.PLAIN_UNIFORM_T, 0),
               ("vanilla_direct", S.VANILLA_DIRECT, 0))
    out = {"workload": "infinite medium sigma_s 10, sigma_a 0.01, point emitter and sensor 3 TMFP apart, "
                       "one gate bin, K=400", "seeds": seeds, "paths_per_render": paths}
    cases = [(0.0, 0.3, gate, paths) for gate in ((0.35, 0.37), (0.6, 0.62), (1.2, 1.24))]
    cases += [(0.7, 1.0, gate, paths) for gate in ((1.5, 1.55), (3.0, 3.1), (6.0, 6.2))]
    # 4x the paths on the isotropic gates: the ratio holds as MSE falls as 1/N
    cases += [(0.0, 0.3, gate, 4 * paths) for gate in ((0.35, 0.37), (0.6, 0.62), (1.2, 1.24))]
    for g, sep, (t0, t1), n_paths in cases:
        sc = S.infinite_scene(10.0, 0.01, g, separation=sep, n_bins=1, t_min=t0, t_max=t1)
        est, tim = {}, {}
        for name, m, fl in methods:
            acc, ts = [], []
            for s_ in range(seeds):
                sp = S.Sampling(seed=900 + s_, paths_per_element=n_paths, max_bounces=400, method=m, flags=fl)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                h = ctx.render(sc, sp)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e-3)
                acc.append(float(h.reshape(-1)[0]))
            est[name], tim[name] = np.array(acc), statistics.median(ts)
        ref = float(np.median(np.concatenate([est["darts"], est["plain_uniform_t"]])))
        res = {"g": g, "separation": sep, "gate": [t0, t1], "paths_per_render": n_paths,
               "reference_median": ref}
        for name, *_ in methods:
            e = est[name]
            iqr = float(np.subtract(*np.percentile(e, [75, 25])))
            d2 = (e - ref) ** 2
            res[name] = {"seconds_per_render": tim[name], "iqr": iqr, "mse_mean": float(d2.mean()),
                         "mse_median": float(np.median(d2))}
        dd = res["darts"]
        for name, *_ in methods[1:]:
            b = res[name]
            res[f"ratio_{name}_over_darts"] = {
                "iqr2_time": (b["iqr"] ** 2 * b["seconds_per_render"]) /
                             max(dd["iqr"] ** 2 * dd["seconds_per_render"], 1e-300),
                "mse_median_time": (b["mse_median"] * b["seconds_per_render"]) /
                                   max(dd["mse_median"] * dd["seconds_per_render"], 1e-300)}
        out[f"g{g:g}_gate_{t0:g}_{t1:g}" + ("" if n_paths == paths else f"_paths{n_paths}")] = res
    return out


def two_peak_response(ctx, S, torch, seeds=16, spp=64):
    """Fig. 7 on the camera box: a temporal response W with two peaks (t = 5
    and 9) over 64 bins on [0, 16).  DARTS samples each path's bin from W;
    the baselines bin every sample by its time.  Reported: MSE x time of the
    W-weighted image sum_b W_b h_b (pooled mean of DARTS and uniform-temporal
    as reference), and the fraction of samples rejected by a zero weight."""
    import numpy as np
    sc = S.box_camera_scene(seed=0, n_bins=64, t_max=16.0)
    t = (np.arange(64) + 0.5) * 0.25
    w = np.exp(-0.5 * ((t - 5.0) / 0.4) ** 2) + np.exp(-0.5 * ((t - 9.0) / 0.6) ** 2)
    w[w < 1e-3] = 0.0
    sc.gate.weights = [float(x) for x in w]
    wt = torch.tensor(w, dtype=torch.float64, device="cuda")
    methods = (("darts", S.DARTS), ("plain_uniform_t", S.PLAIN_UNIFORM_T), ("vanilla_direct", S.VANILLA_DIRECT))
    out = {"workload": "box camera 64x64, 64 bins on [0,16), W = two Gaussian peaks (5 +- 0.4, 9 +- 0.6) "
                       "cut below 1e-3, K=50", "seeds": seeds, "spp": spp}
    imgs, T = {}, {}
    for name, m in methods:
        acc, ts = [], []
        for s_ in range(seeds):
            sp = S.Sampling(seed=501 + s_, paths_per_element=spp, max_bounces=50, method=m,
                            flags=S.FLAG_REBUILD_TABLE if m == S.DARTS else 0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            h = ctx.render(sc, sp)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
            acc.append((h * wt).sum(-1).reshape(-1))
            if s_ == 0:
                st = ctx.stats()
                out.setdefault("rejected_fraction", {})[name] = st["rejected"] / max(st["samples"], 1)
        imgs[name] = torch.stack(acc)
        T[name] = statistics.median(ts)
    ref = torch.cat([imgs["darts"], imgs["plain_uniform_t"]]).mean(0)
    for name, _ in methods:
        d = imgs[name] - ref
        mse = (d * d).mean(1)
        out[name] = {"seconds_per_render": T[name], "mse_mean": float(mse.mean()), "mse_median": float(mse.median())}
    for base in ("plain_uniform_t", "vanilla_direct"):
        out[f"ratio_{base}_over_darts"] = {
            "mse_mean_time": (out[base]["mse_mean"] * out[base]["seconds_per_render"]) /
                             max(out["darts"]["mse_mean"] * out["darts"]["seconds_per_render"], 1e-300),
            "mse_median_time": (out[base]["mse_median"] * out[base]["seconds_per_render"]) /
                               max(out["darts"]["mse_median"] * out["darts"]["seconds_per_render"], 1e-300)}
    return out


def batched_compare(ctx, S, torch, reps=5):
    """256 independent slab media with uneven budgets (2^U[12,20] paths,
    128 bins): one graph-captured persistent launch, in the shape the
    project's autotuner picks (block size, work items per CTA share), vs one
    launch per medium (each in its own tuned shape would cost 256 tunings:
    the per-medium launches use the default shape)."""
    media = S.batched_media(n_media=256, seed=0)
    scenes = [m[0] for m in media]
    samplings = [m[1] for m in media]
    total = sum(sp.paths_per_element for sp in samplings)
    outs = [torch.empty(sc.gate.n_bins, dtype=torch.float64, device="cuda") for sc in scenes]
    t_tune = time.perf_counter()
    tuned = ctx.autotune_batch(scenes, samplings, outs)
    t_tune = time.perf_counter() - t_tune
    # the tuned batch shape; single renders (the per-medium loop) in the default shape
    ctx.set_launch_config(batch_block=tuned["batch_block"], batch_items=tuned["batch_items"])
    ctx.render_batch(scenes, samplings, outs=outs)
    ctx.render_batch(scenes, samplings, outs=outs)
    torch.cuda.synchronize()

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    t_batch = timed(lambda: ctx.render_batch(scenes, samplings, outs=outs), reps)
    events = ctx.stats()  # of the last batched launch
    singles = [torch.empty(sc.gate.n_bins, dtype=torch.float64, device="cuda") for sc in scenes]

    def loop():
        for sc, sp, o in zip(scenes, samplings, singles):
            ctx.render(sc, sp, out=o)

    loop()
    t_loop = timed(loop, 2)
    ctx.set_launch_config()
    return {"media": len(scenes), "paths": total, "ms_batched_graph": t_batch,
            "tuned_shape": {"batch_block": tuned["batch_block"], "batch_items": tuned["batch_items"],
                            "tuning_s": t_tune},
            "ms_one_launch_per_medium": t_loop, "paths_per_s_batched": total / (t_batch * 1e-3),
            "paths_per_s_per_medium_launches": total / (t_loop * 1e-3),
            "speedup": t_loop / t_batch, "events_per_launch": events,
            "vertices_per_s_batched": events["vertices"] / (t_batch * 1e-3),
            "workload": "256 slab media: sigma_s log-uniform [0.1,10], albedo U[0.5,0.999], "
                        "g U[-0.3,0.9], side U[0.5,4], budgets 2^U[12,20], 128 bins, K=50, M=8"}


def frames_in_flight(ctx, S, torch, sc, sp, N, workload, frames=60, calls=10, reps=5):
    """Throughput of a frame sequence (video rendering) through
    darts_render_frames with 1, 2 and 3 frames in flight: frame i runs on
    lane i mod n (a stream of its own), so that a frame's tail (a few long
    paths on a few SMs) overlaps the next frame's start.  `calls` calls of
    `frames` frames each, into `frames` distinct 16 MiB outputs; no L2 flush
    between frames (the lanes run concurrently), the 1-lane row measured the
    same way for the ratio."""
    prep = ctx.prepare(sc, sp)
    outs = [torch.empty(S.histogram_shape(sc), dtype=torch.float64, device="cuda") for _ in range(frames)]
    rows = {}
    for n in (1, 2, 3):
        def run(k):
            for c in range(k):
                prep.render_frames(outs, path_offset=c * frames * N, in_flight=n)

        run(2)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run(calls)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / (frames * calls))
        ms = statistics.median(ts)
        rows[str(n)] = {"ms_per_frame": ms, "paths_per_s": N / (ms * 1e-3)}
    ctx.sync()
    del outs
    for r in rows.values():
        r["vs_one_lane"] = rows["1"]["ms_per_frame"] / r["ms_per_frame"]
    return {"workload": workload, "frames": frames * calls, "call": "darts_render_frames",
            "lanes": rows, "note": "throughput, not the latency of a frame; median of %d repetitions" % reps}


def differentiable_step(ctx, S, torch, flush, reps=10):
    """The differentiable configuration: the unit-cube medium seen by a 32x32
    camera, 256 bins, 2^20 paths (1024 per pixel); L2 loss against a target
    rendered at (sigma_s, sigma_a, g) = (1.3, 0.02, 0.6), gradient at
    (1.0, 0.01, 0.7).  A gradient step is the forward render, the loss
    weights 2 (h - target) and the path-replay adjoint pass with an
    independent seed; the forward render alone is timed beside it."""
    import dataclasses
    sc = S.cube_camera_scene(32, 32)
    star = dataclasses.replace(sc, medium=dataclasses.replace(sc.medium, sigma_s=1.3, sigma_a=0.02, g=0.6))
    sp = S.Sampling(seed=0, paths_per_element=1024)
    spa = dataclasses.replace(sp, seed=1)
    n = S.total_paths(sc, sp)
    target = ctx.render(star, sp)
    h = torch.empty_like(target)
    grad = [None]

    def forward():
        ctx.render(sc, sp, out=h)

    def gradient_step():
        ctx.render(sc, sp, out=h)
        grad[0] = ctx.adjoint(sc, spa, (2.0 * (h - target)).reshape(-1))

    for _ in range(3):
        gradient_step()
    torch.cuda.synchronize()
    tf, _, _ = time_steps(ctx, torch, forward, reps, flush, kernel_timing=False)
    tg, _, _ = time_steps(ctx, torch, gradient_step, reps, flush, kernel_timing=False)
    mf, mg = statistics.median(tf), statistics.median(tg)
    g = grad[0].cpu().tolist()
    return {"workload": "32x32 pinhole view of the unit-cube medium (sigma_s 1, sigma_a 0.01, g 0.7), 256 bins, "
                        "2^20 paths (1024 spp), K=50; L2 loss against a render at (1.3, 0.02, 0.6)",
            "paths": n, "ms_forward": mf, "ms_gradient_step": mg, "ms_adjoint": mg - mf,
            "adjoint_over_forward": (mg - mf) / mf, "gradient_steps_per_s": 1e3 / mg,
            "adjoint_paths_per_s": n / ((mg - mf) * 1e-3), "dL_dsigma_s_sigma_a_g": g}


def time_steps(ctx, torch, step, steps, flush, kernel_timing=True, finish=None):
    """CUDA-event time of each step (L2 flushed before each), the path
    kernel's own time and the summed event counts.  finish() (the last
    exchange of a pipelined multi-rank loop) runs inside the last step."""
    step_ms, kern_ms, stats_acc = [], [], {}
    for i in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        if finish is not None and i == steps - 1:
            finish()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if kernel_timing:
            kern_ms.append(ctx.last_kernel_ms())
        for k, v in ctx.stats().items():
            stats_acc[k] = stats_acc.get(k, 0) + v
    return step_ms, kern_ms, {k: v / steps for k, v in stats_acc.items()}


def mse_time_spheres(ctx, S, torch, seeds=16, spps=(64, 256)):
    """MSE x time on the largest configuration (512x512 camera, 32 spheres,
    two emitters, 1000 bins, K = 100): DARTS, full-gate DARTS, the plain
    uniform-temporal tracer, the vanilla tracer, and DARTS without EDA
    directions and with EDA at surface vertices, `seeds` seeds at 64 and
    256 spp.  The reference is the path-weighted mean of every DARTS and
    uniform-temporal render (both unbiased; 160x the paths of one 64-spp
    render), formed on the device in a first pass; a second pass re-renders
    each seed (deterministic) and takes its MSE over all pixels and bins.
    Also one-bin gates on the same scene (the paper's time-gated regime).
    ratio = (MSE x time)_base / (MSE x time)_darts with the median render
    time (table build + trace, CUDA events)."""
    sc = S.spheres_camera_scene(seed=0)
    methods = (("darts", S.DARTS, 0), ("darts_full_gate", S.DARTS_FULL_GATE, 0),
               ("plain_uniform_t", S.PLAIN_UNIFORM_T, 0), ("vanilla_direct", S.VANILLA_DIRECT, 0),
               ("darts_no_eda", S.DARTS, S.FLAG_NO_EDA), ("darts_surface_eda", S.DARTS, S.FLAG_SURFACE_EDA))
    out = {"workload": "512x512 spheres frame of the benchmark, 1000 bins on [0,20), K=100", "seeds": seeds}

    def render(scene, m, fl, spp, seed, buf):
        sp = S.Sampling(seed=seed, paths_per_element=spp, max_bounces=100, method=m,
                        flags=fl | (S.FLAG_REBUILD_TABLE if m in (S.DARTS, S.DARTS_FULL_GATE) else 0))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.render(scene, sp, out=buf)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    def compare(scene, label, spps_, seed0):
        shape = S.histogram_shape(scene)
        buf = torch.empty(shape, dtype=torch.float64, device="cuda")
        ref = torch.zeros(shape, dtype=torch.float64, device="cuda")
        wsum = 0.0
        for spp in spps_:  # pass 1: the pooled reference
            for name, m, fl in methods[:3:2]:
                for s_ in range(seeds):
                    render(scene, m, fl, spp, seed0 + s_, buf)
                    ref.add_(buf, alpha=float(spp))
                    wsum += spp
        ref.div_(wsum)
        res = {"reference_paths_per_pixel": int(wsum)}
        for spp in spps_:  # pass 2: per-seed MSE
            rows = {}
            for name, m, fl in methods:
                mse, ts = [], []
                for s_ in range(seeds):
                    ts.append(render(scene, m, fl, spp, seed0 + s_, buf))
                    buf.sub_(ref)
                    mse.append(float(torch.mean(buf * buf)))
                mse.sort()
                rows[name] = {"seconds_per_render": statistics.median(ts),
                              "mse_mean": statistics.fmean(mse), "mse_median": statistics.median(mse)}
            for base in ("plain_uniform_t", "vanilla_direct", "darts_full_gate", "darts_no_eda", "darts_surface_eda"):
                b, d = rows[base], rows["darts"]
                rows[f"ratio_{base}_over_darts"] = {
                    "mse_mean_time": b["mse_mean"] * b["seconds_per_render"] /
                                     max(d["mse_mean"] * d["seconds_per_render"], 1e-300),
                    "mse_median_time": b["mse_median"] * b["seconds_per_render"] /
                                       max(d["mse_median"] * d["seconds_per_render"], 1e-300)}
            b, d = rows["plain_uniform_t"], rows["darts_full_gate"]
            rows["ratio_plain_uniform_t_over_darts_full_gate"] = {
                "mse_mean_time": b["mse_mean"] * b["seconds_per_render"] /
                                 max(d["mse_mean"] * d["seconds_per_render"], 1e-300),
                "mse_median_time": b["mse_median"] * b["seconds_per_render"] /
                                   max(d["mse_median"] * d["seconds_per_render"], 1e-300)}
            res[f"spp_{spp}"] = rows
        del buf, ref
        out[label] = res

    compare(sc, "transient_1000_bins", spps, 1001)
    for t0, t1 in ((6.0, 6.25), (10.0, 10.25)):
        g = S.spheres_camera_scene(seed=0, n_bins=1)
        g.gate.t_min, g.gate.t_max = t0, t1
        compare(g, f"gate_{t0:g}_{t1:g}", spps, 2001)
    return out


def roofline(per, kms, workload, traffic_workload=None, paths=None):
    """Algorithmic FP32 work of one launch of the path kernel over its
    measured duration, against the FP32 pipe peak derived from the SM count,
    lanes and the measured maximum clock.  Work per vertex comes from the
    oracle's op-count summary of the same workload; vertices from the
    launch's own event counts."""
    # the 256x256 profiling case is the 512x512 scene: its op counts per vertex
    w = algorithmic_work("spheres_512" if workload == "spheres_256" else workload)
    clock_mhz = measured_peaks().get("sm_max_mhz", 2070.0)
    peak_fp32 = SM_COUNT * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    peak_mufu = SM_COUNT * MUFU_PER_SM_CLK * clock_mhz * 1e6 / 1e12
    out = {"bound": "alu", "achieved": None, "peak": peak_fp32, "unit": "TFLOP/s", "frac": None,
           "traffic": profiled_traffic(traffic_workload or workload, paths) if paths else None,
           "kernel": "trace_kernel (persistent path kernel)", "kernel_ms": kms,
           "peak_note": f"derived nominal: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                        f"{clock_mhz:.0f} MHz (measured max SM clock)",
           "vertices_per_launch": per.get("vertices"),
           "events_per_launch": {k: per[k] for k in ("paths", "vertices", "connections_nonempty", "distance_steps",
                                                     "fp64_ellipse", "fp64_phi") if k in per}}
    if w is None or not kms:
        out["note"] = "no op-count summary for this workload"
        return out
    flops = w["flops_per_vertex"] * per["vertices"]
    special = w["special_per_vertex"] * per["vertices"]
    out.update({"achieved": flops / (kms * 1e-3) / 1e12, "flops_per_launch": flops,
                "work_per_vertex": {"flops": w["flops_per_vertex"], "special": w["special_per_vertex"],
                                    "int": w["int_per_vertex"], "source": "profiles/op_counts.md"},
                "special_frac": special / (kms * 1e-3) / 1e12 / peak_mufu})
    out["frac"] = out["achieved"] / peak_fp32
    return out


def time_workload(ctx, S, torch, name, flush, steps):
    """Compact timing of a secondary workload: paths/s, step and kernel ms,
    FP32 fraction."""
    sc, sp, N = make_workload(name, S)
    prep = ctx.prepare(sc, sp)
    h = torch.empty(S.histogram_shape(sc), dtype=torch.float64, device="cuda")
    ctx.autotune(sc, sp)
    for _ in range(3):
        prep.render(out=h)
    torch.cuda.synchronize()
    ctx.set_kernel_timing(True)
    st, kt, per = time_steps(ctx, torch, lambda: prep.render(out=h), steps, flush)
    ctx.set_kernel_timing(False)
    launch = ctx.launch_config()
    ctx.set_launch_config()
    t = statistics.fmean(st)
    roof = roofline(per, statistics.fmean(kt), name)
    del h
    return {"paths_per_step": N, "ms_per_step": t, "paths_per_s": N / (t * 1e-3),
            "kernel_ms": roof["kernel_ms"], "fp32_frac": roof["frac"],
            "launch": {"block": launch["block"], "chunk": launch["chunk"]}}


def run_studies(ctx, S, torch, flush, sc, sp, N, path):
    """Every side study, written to `path` (one JSON object)."""
    out = {}
    sc16, sp16 = S.cube_workload(paths=1 << 16, seed=0)
    sp16.flags |= S.FLAG_REBUILD_TABLE
    for _ in range(3):
        ctx.render(sc16, sp16)
    torch.cuda.synchronize()
    t16, _, _ = time_steps(ctx, torch, lambda: ctx.render(sc16, sp16), 20, flush, kernel_timing=False)
    out["cube_as_configured_2e16"] = {"paths": 1 << 16, "ms_per_render": statistics.median(t16),
                                      "paths_per_s": (1 << 16) / (statistics.median(t16) * 1e-3)}
    cdf = ctx.build_table(sc, sp)
    ctx.set_kernel_timing(True)
    tt, kt, _ = time_steps(ctx, torch, lambda: ctx.build_table(sc, sp, out=cdf), 20, flush)
    ctx.set_kernel_timing(False)
    out["table_build"] = {"kernel_ms": statistics.median(kt), "call_ms": statistics.median(tt),
                          "bytes": cdf.numel() * 4}
    out["mse_time_spheres_512"] = mse_time_spheres(ctx, S, torch)
    out["mse_time_box_camera"] = mse_time_camera(ctx, S, torch)
    out["mse_time_gated"] = mse_time_gated(ctx, S, torch)
    out["mse_time_gated_dense"] = mse_time_gated_dense(ctx, S, torch)
    out["two_peak_response"] = two_peak_response(ctx, S, torch)
    out["mse_time_cube"] = mse_time(ctx, S, torch)
    out["batched"] = batched_compare(ctx, S, torch)
    out["differentiable_32x32"] = differentiable_step(ctx, S, torch, flush)
    scb, spb, Nb = make_workload("box_camera", S)
    out["frames_in_flight_box_camera"] = frames_in_flight(ctx, S, torch, scb, spb, Nb, "the 64x64 box frame")
    out["frames_in_flight_cube_2e16"] = frames_in_flight(
        ctx, S, torch, sc16, sp16, 1 << 16, "the unit cube as configured, 2^16 paths per render")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_env()
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi, scenes as S, sharding

    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    ctx = capi.Context(local)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    if args.only in ("batched", "differentiable"):
        run = {"batched": lambda: batched_compare(ctx, S, torch),
               "differentiable": lambda: differentiable_step(ctx, S, torch, flush)}[args.only]
        res = run()
        if rank == 0:
            print(json.dumps({"only": args.only, **res}), flush=True)
        ctx.close()
        if pg is not None:
            pg.destroy_process_group()
        return 0
    sc, sp, N = make_workload(args.workload, S)
    camera = sc.sensor.kind == S.SENSOR_PINHOLE
    offset = sharding.path_offset(rank, N)
    prepared = ctx.prepare(sc, sp)  # structs marshalled once, as a renderer loop would
    # under torchrun the all-reduce of step k - 1 runs while step k renders
    pipe = sharding.PipelinedCombine(
        lambda: torch.zeros(S.histogram_shape(sc), dtype=torch.float64, device="cuda"), ws)

    def step():
        hist = pipe.begin_step()
        prepared.render(out=hist, path_offset=offset)
        pipe.end_step(hist)

    # block size and path-counter chunk of the path kernel, tuned on this workload
    if args.launch:
        b_, c_ = (int(x) for x in args.launch.split(","))
        ctx.set_launch_config(block=b_, chunk=c_)
    else:
        ctx.autotune(sc, sp)
    launch = ctx.launch_config()
    for _ in range(args.warmup):
        step()
    pipe.finish()
    torch.cuda.synchronize()
    ctx.set_kernel_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms, kern_ms, per = time_steps(ctx, torch, step, args.steps, flush, finish=pipe.finish)
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ctx.set_kernel_timing(False)
    ctx.sync()

    t_step = sum(step_ms) / len(step_ms)
    if pg is not None:
        tt = torch.tensor([t_step], dtype=torch.float64, device="cuda")
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_step = float(tt.item())
    value = ws * N / (t_step * 1e-3)
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0
    K = args.steps
    kms = statistics.fmean(kern_ms)
    roof = roofline(per, kms, args.workload, paths=N)
    if args.only == "timed":
        print(json.dumps({"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": ws,
                          "steps": K, "warmup": args.warmup, "ms_per_step": t_step,
                          "config": {"workload": args.workload, "launch": launch}, "roofline": roof,
                          "note": "timed steps only"}), flush=True)
        ctx.close()
        return 0
    del pipe
    torch.cuda.empty_cache()

    # ---- end to end through the C ABI with host buffers: queued host renders
    # (darts_render_host_async), the copy of frame i back to pinned host
    # memory overlapping the render of frame i + 1; every frame's histogram
    # reaches the host
    shape = S.histogram_shape(sc)
    hh = [torch.empty(shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    for h_ in hh:
        h_.zero_()  # first touch of the pinned pages, outside the timed region
    ne = max(4, min(K, 30))
    # warm both calls: the context allocates its device histograms (two for
    # the queued call, one for the synchronous one) at their first use
    prepared.render_host(hh[0])
    for i in range(2):
        prepared.render_host_async(hh[i])
    ctx.sync()
    # the host link's bandwidth for one frame's histogram (a plain copy), the
    # bound of the queued call when the copy outlasts the render
    dev_h = torch.zeros(shape, dtype=torch.float64, device="cuda")
    t_copy = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh[1].copy_(dev_h, non_blocking=True)
        torch.cuda.synchronize()
        t_copy.append(time.perf_counter() - t0)
    d2h_gbs = hh[1].numel() * 8 / min(t_copy) / 1e9
    del dev_h
    # five repetitions of ne frames each, the median kept: the copies share
    # the host link with other work on the machine, and a repetition now and
    # then loses one copy's length to it
    t_async, t_sync = [], []
    for rep in range(5):
        te = time.perf_counter()
        for i in range(ne):
            prepared.render_host_async(hh[i % 2], path_offset=(rep * ne + i) * N)
        ctx.sync()
        t_async.append(time.perf_counter() - te)
        # the synchronous call (render, copy back, synchronise per frame) beside it
        ts_ = time.perf_counter()
        for i in range(ne):
            prepared.render_host(hh[0], path_offset=(rep * ne + i) * N)
        t_sync.append(time.perf_counter() - ts_)
    te, ts_ = statistics.median(t_async), statistics.median(t_sync)
    cs, keep = capi.to_c_scene(sc)
    import ctypes
    h2d = (ctypes.sizeof(cs) + ctypes.sizeof(capi.darts_sampling)
           + len(sc.emitters) * ctypes.sizeof(capi.darts_emitter) + 40 * len(sc.geometry.spheres))
    e2e = {"value": N * ne / te, "unit": "paths/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": hh[0].numel() * 8, "frames": ne, "repetitions": 5,
           "ms_per_frame_each": [round(1e3 * t / ne, 3) for t in t_async],
           "d2h_gbs": round(d2h_gbs, 1), "copy_ms_per_frame": round(hh[0].numel() * 8 / d2h_gbs / 1e6, 3),
           "synchronous_value": N * ne / ts_,
           "call": "darts_render_host_async (queued; one darts_sync after the last frame); "
                   "synchronous_value: darts_render_host"}
    del hh
    ctx.sync()
    # the device histograms of the host renders are the context's: released
    # with the context below

    secondary = {}
    for other in ("box_camera", "cube"):
        if other != args.workload:
            secondary[other] = time_workload(ctx, S, torch, other, flush,
                                             200 if other == "box_camera" else 20)
    if args.studies:
        run_studies(ctx, S, torch, flush, sc, sp, N, args.studies)
    cpu = cpu_baseline(args.workload) if ws == 1 else None

    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                       "paths_per_gpu_per_step": N,
                       "launch": {"block": launch["block"], "chunk": launch["chunk"],
                                  "source": "--launch" if args.launch else "darts_autotune on this workload"},
                       "grid": "one CTA per SM (persistent)",
                       "l2": "256 MiB buffer written between timed steps (flush); histogram of "
                             "%.3f GB per step" % (math.prod(S.histogram_shape(sc)) * 8e-9),
                       "parallelism": f"path-id shards x{ws}, FP64 histogram all-reduce of step k-1 "
                                      f"overlapped with the render of step k" if ws > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 2 * K, "clocks": clk, "wall_s_timed_region": wall,
            "secondary": secondary}
    if args.studies:
        line["studies"] = args.studies
    print(json.dumps(line), flush=True)
    ctx.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
