"""Per-path comparison of GPU decision traces with the oracle's (shared by the
GPU parity tests)."""
import numpy as np

import oracle as O

NEAR_TIE = 1e-3
REL_PATH = 1e-4
# FP32 relative error of path lengths and window bounds (about seven units
# of 2^-24): a connection whose window S_hi - S_lo is narrow compared with
# the length L + S_hi it is measured against carries that error magnified by
# cond = (L + S_hi) / (S_hi - S_lo), the oracle's per-path conditioning number.
COND_EPS = 4e-7
# a decision this close to its threshold is a tie at FP32 resolution
EXACT_TIE = 1e-6
# In scenes with surfaces a surface vertex's direct connection is kept only
# when its path time falls in the path's bin; that test is not part of the
# decision record.  After tens of vertices the FP32 position and length
# carry errors of order 1e-5 relative, so a path that met such a test (or
# any decision) within SURFACE_TIE of its threshold may keep a connection on
# one side and drop it on the other with identical traces: it is a tie.
SURFACE_TIE = 1e-5
# the GPU builds its own FP32 direction table: its bin masses may differ from
# the oracle's by up to 2e-6 (asserted by the table parity test; measured
# <= 9e-7), which moves the throughput of a path by at most half that times
# the oracle's per-path table sensitivity (two CDF entries per p_EDA)
TABLE_EPS = 1e-6
# When the GPU renders with the oracle's own table rounded to FP32
# (Context.load_table), a bin mass differs from the oracle's by at most one
# FP32 unit of a CDF value below 1 (2^-24), half of which multiplies the
# per-path table sensitivity as above.
SHARED_TABLE_EPS = 3e-8


def share_oracle_table(ctx, sc, sp):
    """Install the oracle's FP64 direction table, rounded to FP32, as the GPU
    context's table for this scene: both sides then sample directions from
    the same table data (the oracle in FP64, the GPU in FP32), and the
    GPU's own quadrature drops out of the per-path comparison.  Renders and
    debug traces that follow must not set FLAG_REBUILD_TABLE.  Returns the
    oracle table (for O.trace_paths(cdf=...))."""
    return install_table(ctx, sc, sp, O.build_table(sc, sp))


def install_table(ctx, sc, sp, cdf):
    """Install the FP64 table cdf [rows][n_mu + 1], rounded to FP32, as the
    GPU context's table for this scene; returns cdf."""
    import torch
    from paper_2402_03106_gb300 import capi
    rows, nb1 = cdf.shape
    t = np.ones((rows, capi.darts_table_row_stride(sp.table_n_mu)), np.float32)
    t[:, :nb1] = cdf.astype(np.float32)
    ctx.load_table(sc, sp, torch.from_numpy(t).to(ctx._dev()))
    return cdf


def plateau_table(rows, n_mu, seed, zero_frac=0.6):
    """A direction table whose rows are CDFs with runs of zero-probability
    bins (plateaus), including leading and trailing ones: every bin density
    is drawn, most are set to zero, and each row is normalised in FP64.
    Exercises the inverse-CDF search where many bins share one CDF value."""
    rng = np.random.default_rng(seed)
    out = np.empty((rows, n_mu + 1))
    for r in range(rows):
        d = rng.random(n_mu) * (rng.random(n_mu) >= zero_frac)
        if r % 4 == 1:
            d[: n_mu // 3] = 0.0  # leading plateau at 0
        if r % 4 == 2:
            d[-n_mu // 3:] = 0.0  # trailing plateau at 1
        if r % 4 == 3:
            d[:] = 0.0
            d[rng.integers(0, n_mu, 3)] = 1.0  # three bins carry everything
        if d.sum() == 0.0:
            d[rng.integers(0, n_mu)] = 1.0
        c = np.concatenate(([0.0], np.cumsum(d)))
        out[r] = c / c[-1]
        out[r, -1] = 1.0
    return out


def report(name, same, rel, ref, tol, rel_tol=REL_PATH):
    """Summary of one per-path comparison: paths whose traces agree, how many
    of them differ by more than the plain tolerance, the worst relative
    error, and how many needed a conditioning allowance.  Appended as one
    JSON line to $DARTS_PARITY_REPORT when that is set."""
    import json
    import os
    ok = same & ((ref["flags"] & O.FLAG_NEAR_DEGENERATE) == 0)
    r = rel[ok]
    out = {"test": name, "paths": int(len(same)), "same_trace": int(same.sum()),
           "beyond_1e-4": int(np.sum(r > rel_tol)), "frac_beyond_1e-4": float(np.mean(r > rel_tol)) if len(r) else 0.0,
           "worst_rel": float(r.max()) if len(r) else 0.0,
           "worst_path": int(np.nonzero(ok)[0][np.argmax(r)]) if len(r) else -1,
           "needing_allowance": int(np.sum(tol[ok] > rel_tol)), "near_degenerate": int(np.sum(same & ~ok))}
    path = os.environ.get("DARTS_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(out) + "\n")
    return out


def compare_paths(gpu, ref, K):
    """Return (same_trace mask, rel error array, report dict)."""
    gb = gpu["bin"].cpu().numpy()
    gn = gpu["nvert"].cpu().numpy()
    gd = gpu["decisions"].cpu().numpy()
    gc = gpu["contrib"].cpu().numpy().astype(np.float64)
    n = len(gb)
    assert np.array_equal(gb, ref["bin"]), "bin assignment differs"
    same = np.zeros(n, bool)
    first_diff = np.full(n, -1)
    for i in range(n):
        nv = ref["nvert"][i]
        if gn[i] == nv and np.array_equal(gd[i, :nv], ref["decisions"][i, :nv]):
            same[i] = True
        else:
            m = min(gn[i], nv)
            diff = np.nonzero(np.any(gd[i, :m] != ref["decisions"][i, :m], axis=1))[0]
            first_diff[i] = diff[0] if len(diff) else m - 1
    rc = ref["contrib"]
    rel = np.abs(gc - rc) / np.maximum(np.abs(rc), 1e-300)
    rel[(rc == 0) & (gc == 0)] = 0.0
    flips = np.nonzero(~same)[0]
    margins = np.array([ref["margin"][i, : first_diff[i] + 1].min() for i in flips]) if len(flips) else np.array([])
    return same, rel, dict(flips=flips, margins=margins, first_diff=first_diff)


def displaced_sensitivity(sc, sp, first, n, method, ref, shift=1e-6):
    """Relative change of each path's FP64 contribution when the sensor (or
    camera) and its look-at point move by `shift` (length units).

    Paths that meet surfaces at grazing angles magnify any error of their
    start point (each hit divides it by the cosine of incidence); FP32
    arithmetic injects such errors at every vertex (a few units of 2^-24 of
    the coordinates, i.e. of order 1e-6 over a path), so a path whose FP64
    contribution moves by s under this displacement can differ by about s in
    FP32 as well.  Returns s per path (0 where both are zero)."""
    import copy
    sc2 = copy.deepcopy(sc)
    d = np.array([1.0, -0.7, 0.4]) * shift
    sc2.sensor.pos = tuple(np.asarray(sc.sensor.pos, float) + d)
    sc2.sensor.look_at = tuple(np.asarray(sc.sensor.look_at, float) + d)
    r2 = O.trace_paths(sc2, sp, first, n, method=method)
    c, c2 = ref["contrib"], r2["contrib"]
    s = np.abs(c2 - c) / np.maximum(np.abs(c), 1e-300)
    s[(c == 0) & (c2 == 0)] = 0.0
    return s


def check_paths(gpu, ref, K, rel_tol=REL_PATH, max_flip_frac=0.01, extra_tol=None, table_eps=TABLE_EPS,
                name=None, tie_margin=EXACT_TIE):
    """Flips must sit at a decision the oracle met within NEAR_TIE of its
    threshold.  Flips at an exact tie (margin below FP32 resolution, e.g. a
    bin edge that coincides with a table cell edge, rho = C/S_M = 1/2) may be
    any number; the others at most max_flip_frac of the paths."""
    same, rel, rep = compare_paths(gpu, ref, K)
    n = len(same)
    if len(rep["margins"]):
        assert rep["margins"].max() < NEAR_TIE, f"trace flip away from a tie: {rep['margins']}"
    n_soft = int(np.sum(rep["margins"] >= EXACT_TIE)) if len(rep["margins"]) else 0
    assert n_soft <= max(2, max_flip_frac * n), f"{n_soft} of {n} traces differ away from exact ties"
    nd = (ref["flags"] & O.FLAG_NEAR_DEGENERATE) != 0
    # a path that met an exact tie may have taken the other branch of a
    # decision the trace does not record (the table cell of an EDA sample)
    tie = ref["margin"].min(axis=1) < tie_margin
    ok = same & ~nd & ~tie
    tol = np.maximum(rel_tol, COND_EPS * ref["cond"] + table_eps * ref["tabcond"])
    if extra_tol is not None:
        tol = np.maximum(tol, extra_tol)
    if name is not None:
        report(name, same & ~tie, rel, ref, tol, rel_tol)
    bad = np.nonzero(ok & (rel > tol))[0]
    assert len(bad) == 0, (f"{len(bad)} paths beyond their tolerance: rel {rel[bad][:5]}, "
                           f"tol {tol[bad][:5]}, cond {ref['cond'][bad][:5]}")
    # near-degenerate ellipses (S - C < 2^-12 C) depend on FP32 path state; bound them loosely
    if np.any(same & nd):
        assert rel[same & nd].max() < 1e-2
    return same, rel
