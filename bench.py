#!/usr/bin/env python3
"""Throughput benchmark of the DARTS hot path on GB300.

One step = one pass of the whole path: the elliptical DA direction table is
rebuilt on the GPU, then every path of the step is traced (DA-RIS distance
sampling, EDA/MIS directions, elliptical control vertices) and accumulated
into the time-bin histogram.  The workload is the unit-cube medium
(sigma_s = 1, sigma_a = 0.01, g = 0.7; point emitter at (.5,.5,.1), point
sensor at (.5,.5,.9); 256 bins on [0.8, 6); 50 bounces, 8 RIS candidates,
16x8x256 table) with 2^24 paths per GPU per step.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank traces its own path-id range (weak scaling) and the
per-rank histograms are summed with one FP64 all-reduce per step.  The
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
PATHS_PER_GPU = 1 << 24
WORKLOAD = ("unit-cube medium sigma_s=1 sigma_a=0.01 g=0.7 v=1; isotropic point pulse emitter "
            "(0.5,0.5,0.1) t0=0; point fluence sensor (0.5,0.5,0.9); 256 bins on [0.8,6.0); "
            "K=50 bounces, N_RIS=8, table 16x8x256; 2^24 paths per GPU per step")

# Algorithmic FP32 work of the DARTS step (counted from the equations of the
# stable formulation; add/sub/mul/compare/convert = 1, FMA = 2; special
# functions counted separately as MUFU operations).
FLOPS_PER_VERTEX = 120
FLOPS_PER_CONNECTION = 80
FLOPS_PER_CANDIDATE = 52
FLOPS_PER_DISTANCE_STEP = 30
MUFU_PER_VERTEX = 10
MUFU_PER_CONNECTION = 6
MUFU_PER_CANDIDATE = 5
SM_COUNT = 152
FP32_LANES_PER_SM = 128
MUFU_PER_SM_CLK = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--paths", type=int, default=PATHS_PER_GPU)
    ap.add_argument("--no-mse", action="store_true", help="skip the MSE x time comparison")
    ap.add_argument("--only-timed", action="store_true",
                    help="run only the timed steps (for profiler launch lists)")
    return ap.parse_args()


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
                 "--format=csv,noheader,nounits", "-lms", "100"],
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
    for f in ("trace.cu", "darts_device.cuh", "darts_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2402_03106_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(paths_per_launch: int):
    """DRAM bytes per launch from the committed ncu summary of the trace
    kernel, scaled to this launch, when it was taken on the current source."""
    path = os.path.join(ROOT, "profiles", "darts_trace_kernel_cube.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+-]+)", text)
    m_paths = re.search(r"paths_per_launch:\s*([0-9]+)", text)
    if not (m_hash and m_bytes and m_paths) or m_hash.group(1) != kernel_source_hash():
        return None
    # the DRAM traffic is the fixed table staging and block partials: it does
    # not grow with the number of paths, so it is reported as captured
    return float(m_bytes.group(1))


# ----------------------------------------------------------------------------
def cpu_baseline(paths: int = 1 << 23):
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    sc, sp = S.cube_workload(paths=paths, seed=0)
    cores = os.cpu_count() or 1
    cdf = O.build_table(sc, sp)
    t0 = time.perf_counter()
    O.render(sc, sp, O.ORC_DARTS, cdf=cdf, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": paths / dt, "unit": "paths/s", "cores": cores, "kind": "oracle",
            "sample": f"{paths} paths of the benchmark workload (table prebuilt), FP64 C oracle, "
                      f"{cores} POSIX threads, {dt:.2f} s wall"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    cores = os.cpu_count() or 1
    sample = 1 << 18
    sc, sp = S.cube_workload(paths=sample, seed=0)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cdf = O.build_table(sc, sp)
        O.render(sc, sp, O.ORC_DARTS, cdf=cdf, threads=cores, offset=i * sample)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = sample * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "paths/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("2^24 paths per GPU per step",
                                                    f"{sample} paths per step (bounded CPU sample)")},
            "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} paths per step incl. the table build, "
                                       f"{cores} POSIX threads"},
            "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
def mse_time(ctx, S, torch, n_paths=1 << 20, seeds=16):
    """Efficiency of DARTS against the plain uniform-temporal path tracer (and
    the vanilla direct-connection tracer and the ablations of Fig. 13) at
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
        for base in ("plain_uniform_t", "vanilla_direct", "darts_no_da", "darts_no_eda", "darts_no_da_no_eda"):
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


def batched_compare(ctx, S, torch, reps=5):
    """256 independent slab media with uneven budgets (2^U[12,20] paths,
    128 bins): one graph-captured persistent launch vs one launch per medium."""
    media = S.batched_media(n_media=256, seed=0)
    scenes = [m[0] for m in media]
    samplings = [m[1] for m in media]
    total = sum(sp.paths_per_element for sp in samplings)
    outs = ctx.render_batch(scenes, samplings)
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
    singles = [torch.empty(sc.gate.n_bins, dtype=torch.float64, device="cuda") for sc in scenes]

    def loop():
        for sc, sp, o in zip(scenes, samplings, singles):
            ctx.render(sc, sp, out=o)

    loop()
    t_loop = timed(loop, 2)
    return {"media": len(scenes), "paths": total, "ms_batched_graph": t_batch,
            "ms_one_launch_per_medium": t_loop, "paths_per_s_batched": total / (t_batch * 1e-3),
            "paths_per_s_per_medium_launches": total / (t_loop * 1e-3),
            "speedup": t_loop / t_batch,
            "workload": "256 slab media: sigma_s log-uniform [0.1,10], albedo U[0.5,0.999], "
                        "g U[-0.3,0.9], side U[0.5,4], budgets 2^U[12,20], 128 bins, K=50, M=8"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    ws, rank, local = dist_env()
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi, scenes as S

    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    ctx = capi.Context(local)
    sc, _ = S.cube_workload()
    N = args.paths
    sp = S.Sampling(seed=0, paths_per_element=N, flags=S.FLAG_REBUILD_TABLE)
    B = sc.gate.n_bins
    hist = torch.zeros(B, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    from paper_2402_03106_gb300 import sharding
    offset = sharding.path_offset(rank, N)

    def step():
        ctx.render(sc, sp, out=hist, path_offset=offset)
        sharding.combine(hist, ws)

    tuned_block = ctx.autotune(sc, sp)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.set_kernel_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms = [], []
    stats_acc = {}
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(ctx.last_kernel_ms())
        for k, v in ctx.stats().items():
            stats_acc[k] = stats_acc.get(k, 0) + v
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

    # ---- roofline of the dominant kernel (the persistent path kernel)
    K = args.steps
    per = {k: v / K for k, v in stats_acc.items()}
    flops = (FLOPS_PER_VERTEX * per["vertices"] + FLOPS_PER_CONNECTION * per["connections_nonempty"]
             + (FLOPS_PER_DISTANCE_STEP + 8 * FLOPS_PER_CANDIDATE) * per["distance_steps"])
    mufu = (MUFU_PER_VERTEX * per["vertices"] + MUFU_PER_CONNECTION * per["connections_nonempty"]
            + 8 * MUFU_PER_CANDIDATE * per["distance_steps"])
    kms = statistics.fmean(kern_ms)
    clock_mhz = measured_peaks().get("sm_max_mhz", 2070.0)
    peak_fp32 = SM_COUNT * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12
    peak_mufu = SM_COUNT * MUFU_PER_SM_CLK * clock_mhz * 1e6 / 1e12
    achieved = flops / (kms * 1e-3) / 1e12
    traffic = profiled_traffic(N)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
            "frac": achieved / peak_fp32, "traffic": traffic,
            "kernel": "trace_kernel<DARTS> (persistent path kernel)",
            "kernel_ms": kms, "flops_per_launch": flops,
            "peak_note": f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {clock_mhz:.0f} MHz",
            "mufu_achieved_tops": mufu / (kms * 1e-3) / 1e12, "mufu_peak_tops": peak_mufu,
            "mufu_frac": mufu / (kms * 1e-3) / 1e12 / peak_mufu,
            "events_per_launch": per}

    if args.only_timed:
        print(json.dumps({"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": ws,
                          "steps": K, "warmup": args.warmup, "ms_per_step": t_step,
                          "roofline": roof, "block": tuned_block, "note": "timed steps only"}),
              flush=True)
        ctx.close()
        return 0

    # ---- as configured: 2^16 paths per render (latency-bound)
    sp16 = S.Sampling(seed=0, paths_per_element=1 << 16, flags=S.FLAG_REBUILD_TABLE)
    for _ in range(3):
        ctx.render(sc, sp16)
    torch.cuda.synchronize()
    t16 = []
    for _ in range(20):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.render(sc, sp16)
        e1.record()
        e1.synchronize()
        t16.append(e0.elapsed_time(e1))
    as_conf = {"paths": 1 << 16, "ms_per_render": statistics.median(t16),
               "paths_per_s": (1 << 16) / (statistics.median(t16) * 1e-3)}

    # ---- end to end through the C ABI with host buffers
    hh = torch.zeros(B, dtype=torch.float64).pin_memory()
    ne = max(3, min(args.steps, 20))
    ctx.render_host(sc, sp, hh)
    te = time.perf_counter()
    for i in range(ne):
        ctx.render_host(sc, sp, hh, path_offset=i * N)
    te = time.perf_counter() - te
    cs, keep = capi.to_c_scene(sc)
    import ctypes
    h2d = ctypes.sizeof(cs) + ctypes.sizeof(capi.darts_sampling) + ctypes.sizeof(capi.darts_emitter)
    e2e = {"value": N * ne / te, "unit": "paths/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": B * 8,
           "note": "darts_render_host: scene/sampling structs marshalled into the launches, "
                   "histogram copied back to pinned host memory, stream synchronised per step"}

    mse = None if args.no_mse else mse_time(ctx, S, torch)
    batched = batched_compare(ctx, S, torch)
    cpu = cpu_baseline() if ws == 1 else None

    line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "paths_per_gpu_per_step": N,
                       "block": tuned_block, "grid": "one CTA per SM (persistent)",
                       "l2": "256 MiB buffer written between timed steps (flush)",
                       "parallelism": f"path-id shards x{ws}, FP64 histogram all-reduce" if ws > 1
                       else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 2 * K,
            "clocks": clk, "wall_s_timed_region": wall,
            "as_configured_2e16": as_conf, "mse_time": mse, "batched": batched}
    print(json.dumps(line), flush=True)
    ctx.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
