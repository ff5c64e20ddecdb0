"""GPU per-path parity with one direction table on both sides.

The other parity tests let each side build its own direction table (the GPU
by FP32 quadrature, the oracle by FP64 quadrature) and widen each path's
tolerance by the table difference.  Here the oracle's FP64 table, rounded
to FP32, is installed in the GPU context (darts_load_table, the path for a
table tabulated offline as the paper does in Sec. 5.1): both sides then
sample directions from the same table data, and the per-path bar is the
plain 1e-4 relative, widened only where the oracle's conditioning numbers
say FP32 cannot hold it (narrow connection windows; one FP32 unit of a CDF
value; grazing surface hits in scenes with walls and spheres).  Each test
also reports how many paths needed such an allowance and its worst path
(a JSON line per test in $DARTS_PARITY_REPORT when that is set).

Nothing of the CUDA path flows into the oracle: the data goes the other way.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_03106_gb300 import scenes as S  # noqa: E402
from parity_util import (REL_PATH, SHARED_TABLE_EPS, SURFACE_TIE, check_paths,  # noqa: E402
                         displaced_sensitivity, install_table, plateau_table, report,
                         share_oracle_table)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi
    c = capi.Context(0)
    yield c
    c.close()


def test_loaded_table_is_the_one_rendered_with(ctx):
    """A loaded table replaces the cached one: a render that uses it equals
    a render with the same table rebuilt only when the tables are equal, and
    FLAG_REBUILD_TABLE restores the GPU's own."""
    sc, sp = S.cube_workload(paths=1 << 16, seed=1)
    own = ctx.build_table(sc, sp)
    h_own = ctx.render(sc, S.Sampling(**{**sp.__dict__, "flags": S.FLAG_REBUILD_TABLE}))
    share_oracle_table(ctx, sc, sp)
    h_shared = ctx.render(sc, sp)
    ctx.load_table(sc, sp, own)
    h_again = ctx.render(sc, sp)
    ctx.sync()
    assert torch.equal(h_again, h_own) or torch.allclose(h_again, h_own, rtol=1e-12, atol=0)
    # the oracle's table is a different (FP64-quadrature) table: some bins move
    assert not torch.equal(h_shared, h_own)
    rel = torch.linalg.norm(h_shared - h_own) / torch.linalg.norm(h_own)
    assert float(rel) < 1e-2


@pytest.mark.parametrize("K", [1, 3, 50])
def test_shared_table_per_path_parity(ctx, K):
    sc, sp = S.cube_workload(paths=1 << 16, seed=2)
    sp.max_bounces = K
    cdf = share_oracle_table(ctx, sc, sp)
    n = 4096
    gpu = ctx.debug_paths(sc, sp, 12345, n)
    torch.cuda.synchronize()
    ref = O.trace_paths(sc, sp, 12345, n, cdf=cdf)
    check_paths(gpu, ref, K, table_eps=SHARED_TABLE_EPS, name=f"shared_table_cube_K{K}")


@pytest.mark.parametrize("ris_m", [8, 4])
@pytest.mark.parametrize("flags", [S.FLAG_NO_DA_DISTANCE, S.FLAG_NO_EDA, S.FLAG_SENSOR_UNIFORM_ONLY,
                                   S.FLAG_IID_CANDIDATES, S.FLAG_EQUIANGULAR, S.FLAG_RESERVOIR])
def test_shared_table_ablation_parity(ctx, flags, ris_m):
    sc, sp = S.cube_workload(paths=1 << 16, seed=6)
    sp.flags = flags
    sp.ris_m = ris_m
    cdf = share_oracle_table(ctx, sc, sp)
    n = 2048
    gpu = ctx.debug_paths(sc, sp, 0, n)
    ref = O.trace_paths(sc, sp, 0, n, cdf=cdf)
    check_paths(gpu, ref, sp.max_bounces, table_eps=SHARED_TABLE_EPS,
                name=f"shared_table_ablation_{flags}_M{ris_m}")


def test_shared_table_dense_medium(ctx):
    sc = S.slab_scene(8.0, 0.05, 0.5, n_bins=64, t_min=0.8, t_max=6.0)
    sp = S.Sampling(seed=9, paths_per_element=1 << 14, max_bounces=50)
    cdf = share_oracle_table(ctx, sc, sp)
    n = 2048
    gpu = ctx.debug_paths(sc, sp, 0, n)
    ref = O.trace_paths(sc, sp, 0, n, cdf=cdf)
    check_paths(gpu, ref, 50, max_flip_frac=0.03, table_eps=SHARED_TABLE_EPS, name="shared_table_dense")


def test_shared_table_full_size_sampled_paths(ctx):
    """2^24 paths in the benchmark's launch configuration with the shared
    table; 2048 sampled paths recomputed one by one by the oracle.  Paths
    whose trace flipped near a tie differ entirely (at most 1 %); every
    other sampled path holds 1e-4 unless its conditioning number allows
    more, and those are counted."""
    sc, sp = S.cube_workload(paths=1 << 24, seed=0)
    cdf = share_oracle_table(ctx, sc, sp)
    stride = (1 << 24) // 2048
    probe, pc, pb = ctx.probe(first=7, stride=stride, count=2048)
    ctx.render(sc, sp, probe=probe)
    ctx.sync()
    ids = 7 + stride * np.arange(2048)
    recs = [O.trace_paths(sc, sp, int(pid), 1, cdf=cdf) for pid in ids]
    c_ref = np.array([r["contrib"][0] for r in recs])
    b_ref = np.array([r["bin"][0] for r in recs])
    cond = np.array([r["cond"][0] for r in recs])
    tabc = np.array([r["tabcond"][0] for r in recs])
    assert np.array_equal(pb.cpu().numpy(), b_ref)
    gc = pc.cpu().numpy().astype(np.float64)
    rel = np.abs(gc - c_ref) / np.maximum(np.abs(c_ref), 1e-300)
    rel[(c_ref == 0) & (gc == 0)] = 0
    tol = np.maximum(REL_PATH, 4e-7 * cond + SHARED_TABLE_EPS * tabc)
    beyond = rel > tol
    assert np.mean(beyond) <= 0.01, np.sort(rel)[-10:]
    fake = {"flags": np.zeros(2048, np.int64)}
    report("shared_table_full_size_2e24", ~beyond, rel, fake, tol)


@pytest.mark.parametrize("scene", ["box_camera", "spheres_512"])
def test_shared_table_camera_scenes(ctx, scene):
    """The two camera workloads of the benchmark at their full resolution,
    2048 paths from the middle of the frame, with the shared table; grazing
    surface hits keep their measured allowance (5x the FP64 change under a
    1e-6 displacement of the camera), which stays the exception.  A
    surface connection's in-bin test is not in the decision record, so a
    path that met any decision within 1e-5 of its threshold is a tie (one
    such path of the box frame keeps a connection in FP32 that the oracle
    drops, 2e-6 from a bin edge after 21 vertices)."""
    if scene == "box_camera":
        sc, sp = S.box_camera_workload(seed=0)
        first = 32 * 64 * 16
    else:
        sc = S.spheres_camera_scene(seed=0)
        sp = S.Sampling(seed=0, paths_per_element=64, max_bounces=100)
        first = 256 * 512 * 64
    cdf = share_oracle_table(ctx, sc, sp)
    n = 2048
    gpu = ctx.debug_paths(sc, sp, first, n)
    ref = O.trace_paths(sc, sp, first, n, cdf=cdf)
    sens = 5.0 * displaced_sensitivity(sc, sp, first, n, S.DARTS, ref)
    check_paths(gpu, ref, sp.max_bounces, extra_tol=sens, table_eps=SHARED_TABLE_EPS,
                name=f"shared_table_{scene}", tie_margin=SURFACE_TIE)
    assert np.count_nonzero(ref["contrib"]) > n // 50
    # the grazing allowance stays the exception: under 2 % of the paths get more than 1e-3
    assert np.mean(sens > 1e-3) < 0.02


@pytest.mark.parametrize("name", ["box_64", "cube_camera_32", "spheres_512"])
def test_shared_table_full_size_frames(ctx, name):
    """The camera workloads at full size in one render call (the benchmark's
    launch), with the oracle's table on the GPU: 2048 sampled paths
    recomputed one by one.  Each path must hold the plain 1e-4, widened only
    by its own FP32 allowance (narrow windows, one FP32 unit of the table,
    5x its FP64 change under a 1e-6 camera displacement for grazing hits);
    paths that met a decision within 1e-5 of its threshold are ties, and
    paths beyond their bound (trace flips near a tie, which the probe does
    not record) may be at most 1 %.  The counts are reported."""
    if name == "box_64":
        sc, sp = S.box_camera_workload(seed=0)
    elif name == "cube_camera_32":
        sc = S.cube_camera_scene(32, 32)
        sp = S.Sampling(seed=0, paths_per_element=1024)
    else:
        sc = S.spheres_camera_scene(seed=0)
        sp = S.Sampling(seed=0, paths_per_element=64, max_bounces=100)
    cdf = share_oracle_table(ctx, sc, sp)
    n = S.total_paths(sc, sp)
    stride = n // 2048
    probe, pc, pb = ctx.probe(first=11, stride=stride, count=2048)
    h = ctx.render(sc, sp, probe=probe)
    ctx.sync()
    del h
    ids = 11 + stride * np.arange(2048)
    recs = [O.trace_paths(sc, sp, int(pid), 1, cdf=cdf) for pid in ids]
    c_ref = np.array([r["contrib"][0] for r in recs])
    b_ref = np.array([r["bin"][0] for r in recs])
    cond = np.array([r["cond"][0] for r in recs])
    tabc = np.array([r["tabcond"][0] for r in recs])
    flags = np.array([r["flags"][0] for r in recs])
    tie = np.array([r["margin"][0].min() < SURFACE_TIE for r in recs])
    sens = np.array([displaced_sensitivity(sc, sp, int(pid), 1, S.DARTS,
                                           {"contrib": np.array([c])})[0] for pid, c in zip(ids, c_ref)])
    assert np.array_equal(pb.cpu().numpy(), b_ref)
    gc = pc.cpu().numpy().astype(np.float64)
    rel = np.abs(gc - c_ref) / np.maximum(np.abs(c_ref), 1e-300)
    rel[(c_ref == 0) & (gc == 0)] = 0
    tol = np.maximum(REL_PATH, np.maximum(4e-7 * cond + SHARED_TABLE_EPS * tabc, 5.0 * sens))
    nd = (flags & O.FLAG_NEAR_DEGENERATE) != 0
    tol[nd] = np.maximum(tol[nd], 1e-2)
    beyond = (rel > tol) & ~tie
    assert np.mean(beyond) <= 0.01, (np.sort(rel[beyond])[-10:], np.count_nonzero(beyond))
    assert np.count_nonzero(c_ref) > 50
    report(f"shared_table_full_size_{name}", ~beyond & ~tie, rel, {"flags": flags}, tol)


@pytest.mark.parametrize("scene", ["cube", "box_camera"])
def test_plateau_table_per_path_parity(ctx, scene):
    """Direction sampling from a table whose rows have runs of zero-probability
    bins (leading, trailing and inner plateaus; rows with three live bins),
    loaded on both sides.  The GPU's inverse-CDF search starts from a coarse
    guide of each row, whose entries coincide on plateaus; the oracle takes
    the first bin whose upper CDF edge exceeds the uniform.  Bins and traces
    must agree path by path, contributions within the shared-table bar."""
    if scene == "cube":
        sc, sp = S.cube_workload(paths=1 << 16, seed=3)
        sp.max_bounces = 50
        first, n = 0, 4096
    else:
        sc, sp = S.box_camera_workload(seed=0)
        first, n = 32 * 64 * 16, 2048
    cdf = install_table(ctx, sc, sp, plateau_table(sp.table_n_rho * sp.table_n_s, sp.table_n_mu, seed=11))
    gpu = ctx.debug_paths(sc, sp, first, n)
    torch.cuda.synchronize()
    ref = O.trace_paths(sc, sp, first, n, cdf=cdf)
    kw = {}
    if scene != "cube":  # grazing surface hits: as in the camera tests above
        kw = {"extra_tol": 5.0 * displaced_sensitivity(sc, sp, first, n, S.DARTS, ref), "tie_margin": SURFACE_TIE}
    check_paths(gpu, ref, sp.max_bounces, table_eps=SHARED_TABLE_EPS, name=f"plateau_table_{scene}", **kw)
    assert np.count_nonzero(ref["contrib"]) > n // 50
