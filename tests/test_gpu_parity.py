"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances:
  * Philox blocks, bin assignment, per-path decision traces: bit-exact
    (a trace may differ only where the oracle met a decision within 1e-3 of
    its threshold -- FP32 and FP64 then legitimately take different sides --
    and on at most 1 % of paths);
  * direction tables: |cdf_gpu - cdf_oracle| <= 2e-6, bin masses too;
  * per-path contributions of paths with identical traces: relative 1e-4;
  * histograms at matched seeds: relative L2 <= 1e-3 and every bin within
    3 standard errors.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_03106_gb300 import scenes as S  # noqa: E402
from parity_util import NEAR_TIE, REL_PATH, check_paths, displaced_sensitivity  # noqa: E402,F401

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


# ---------------------------------------------------------------------------
def test_philox_bit_exact(ctx):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 2 ** 32 - 1
    for seed in (0, 123456789, 2 ** 63 + 5):
        out = ctx.philox(ctr.astype(np.int64), seed).cpu().to(torch.int64).numpy().reshape(-1, 4)
        key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        for i in range(0, 4096, 97):
            assert O.philox([int(x) for x in ctr[i]], key) == out[i].tolist()


TABLE_CASES = [
    S.cube_workload(),
    (S.slab_scene(10.0, 0.1, -0.3, side=4.0, n_bins=128), S.Sampling()),
    (S.slab_scene(0.1, 0.05, 0.9, side=0.5, n_bins=128), S.Sampling()),
    (S.slab_scene(2.0, 0.5, 0.0, side=1.0, n_bins=16), S.Sampling(table_n_rho=5, table_n_s=3, table_n_mu=37)),
]


@pytest.mark.parametrize("case", range(len(TABLE_CASES)))
def test_direction_table_matches_oracle(ctx, case):
    sc, sp = TABLE_CASES[case]
    cdf = ctx.build_table(sc, sp).cpu().numpy().astype(np.float64)
    ref = O.build_table(sc, sp)
    nb = sp.table_n_mu
    # FP32 quadrature and scan against FP64: CDF values and bin masses within
    # 2e-6 (the per-path tolerances rely on the mass bound)
    np.testing.assert_allclose(cdf[:, : nb + 1], ref, atol=2e-6, rtol=0)
    np.testing.assert_allclose(np.diff(cdf[:, : nb + 1], axis=1), np.diff(ref, axis=1), atol=2e-6, rtol=0)
    assert np.all(cdf[:, 0] == 0.0) and np.all(cdf[:, nb] == 1.0)


@pytest.mark.parametrize("K", [1, 3, 50])
def test_darts_per_path_parity(ctx, K):
    sc, sp = S.cube_workload(paths=1 << 16, seed=2)
    sp.max_bounces = K
    n = 4096
    gpu = ctx.debug_paths(sc, sp, 12345, n)
    torch.cuda.synchronize()
    ref = O.trace_paths(sc, sp, 12345, n)
    check_paths(gpu, ref, K)


def test_path_ids_across_the_32_bit_boundary(ctx):
    """Global path ids past 2^32 (a path offset of a long progressive render
    or a high rank): the Philox counter carries the id's high word, DARTS
    bins and camera elements follow the 64-bit id.  2048 paths straddling
    2^32, on the specialised kernel (point sensor) and on the general one
    (a camera frame, whose ids wrap over the pixels with the sample index
    continuing)."""
    first = (1 << 32) - 1000
    sc, sp = S.cube_workload(paths=1 << 16, seed=4)
    sp.max_bounces = 20
    gpu = ctx.debug_paths(sc, sp, first, 2048)
    ref = O.trace_paths(sc, sp, first, 2048)
    check_paths(gpu, ref, sp.max_bounces)
    sc = S.box_camera_scene(seed=0, width=16, height=16, n_bins=128)
    sp = S.Sampling(seed=5, paths_per_element=8, max_bounces=20)
    gpu = ctx.debug_paths(sc, sp, first, 2048)
    ref = O.trace_paths(sc, sp, first, 2048)
    sens = 5.0 * displaced_sensitivity(sc, sp, first, 2048, S.DARTS, ref)
    check_paths(gpu, ref, sp.max_bounces, extra_tol=sens)
    assert np.count_nonzero(ref["contrib"]) > 100


@pytest.mark.parametrize("ris_m", [8, 4])
@pytest.mark.parametrize("flags", [S.FLAG_NO_DA_DISTANCE, S.FLAG_NO_EDA,
                                   S.FLAG_NO_DA_DISTANCE | S.FLAG_NO_EDA, S.FLAG_SENSOR_UNIFORM_ONLY,
                                   S.FLAG_IID_CANDIDATES, S.FLAG_EQUIANGULAR, S.FLAG_RESERVOIR,
                                   S.FLAG_IID_CANDIDATES | S.FLAG_EQUIANGULAR | S.FLAG_RESERVOIR,
                                   S.FLAG_EQUIANGULAR | S.FLAG_NO_DA_DISTANCE])
def test_ablation_per_path_parity(ctx, flags, ris_m):
    """Ablations and RIS variants, on the warp-cooperative RIS (M = 8) and on
    the per-lane RIS (M = 4)."""
    sc, sp = S.cube_workload(paths=1 << 16, seed=6)
    sp.flags = flags
    sp.ris_m = ris_m
    n = 2048
    gpu = ctx.debug_paths(sc, sp, 0, n)
    ref = O.trace_paths(sc, sp, 0, n)
    check_paths(gpu, ref, sp.max_bounces)


def test_darts_per_path_parity_dense_medium(ctx):
    """Many scattering events per path: sigma_s = 8 in a unit cube."""
    sc = S.slab_scene(8.0, 0.05, 0.5, n_bins=64, t_min=0.8, t_max=6.0)
    sp = S.Sampling(seed=9, paths_per_element=1 << 14, max_bounces=50)
    n = 2048
    gpu = ctx.debug_paths(sc, sp, 0, n)
    ref = O.trace_paths(sc, sp, 0, n)
    check_paths(gpu, ref, 50, max_flip_frac=0.03)


@pytest.mark.parametrize("method", [S.PLAIN_UNIFORM_T, S.VANILLA_DIRECT, S.DARTS_FULL_GATE])
def test_baseline_per_path_parity(ctx, method):
    sc, sp = S.cube_workload(paths=1 << 14, seed=4)
    sp.method = method
    n = 4096
    gpu = ctx.debug_paths(sc, sp, 0, n)
    ref = O.trace_paths(sc, sp, 0, n, method=method)
    check_paths(gpu, ref, sp.max_bounces)


def test_ris_variants_histogram_and_unsupported_combinations(ctx):
    from paper_2402_03106_gb300 import capi
    sc, sp = S.cube_workload(paths=1 << 16, seed=31)
    sp.flags = S.FLAG_IID_CANDIDATES | S.FLAG_EQUIANGULAR | S.FLAG_RESERVOIR
    h = ctx.render(sc, sp).cpu().numpy()
    href, _, _ = O.render(sc, sp, O.ORC_DARTS)
    assert np.linalg.norm(h - href) <= 1e-3 * np.linalg.norm(href)
    cam = S.box_camera_scene(width=4, height=4, n_bins=16)
    for call in (lambda: ctx.render(cam, S.Sampling(paths_per_element=4, flags=S.FLAG_RESERVOIR)),
                 lambda: ctx.adjoint(sc, sp, torch.ones(sc.gate.n_bins, dtype=torch.float64)),
                 lambda: ctx.render_batch([sc], [sp])):
        with pytest.raises(capi.DartsError) as ei:
            call()
        assert ei.value.status == 6


@pytest.mark.parametrize("method", [S.DARTS, S.PLAIN_UNIFORM_T, S.VANILLA_DIRECT, S.DARTS_FULL_GATE])
def test_histogram_parity_matched_seeds(ctx, method):
    sc, sp = S.cube_workload(paths=1 << 16, seed=0)
    sp.method = method
    hist, sq = ctx.render(sc, sp, sumsq=True)
    ctx.sync()
    h = hist.cpu().numpy()
    href, sqref, _ = O.render(sc, sp, method)
    per_bin = (1 << 16) / 256 if method == S.DARTS else (1 << 16)
    se = O.standard_error(href, sqref, per_bin)
    l2 = np.linalg.norm(h - href) / np.linalg.norm(href)
    assert l2 < 1e-3, l2
    assert np.all(np.abs(h - href) <= 3 * se + 1e-12 * np.abs(href).max())
    if method == S.DARTS:
        # one commit per DARTS path: the per-path squares are exact.  The
        # baselines square each connection (a path hitting a bin twice is not
        # merged), so their sums of squares are checked only for consistency.
        np.testing.assert_allclose(sq.cpu().numpy(), sqref, rtol=1e-3, atol=1e-12 * sqref.max())
    else:
        assert np.all(sq.cpu().numpy() >= 0) and sq.cpu().numpy().sum() <= 1.0001 * sqref.sum()


@pytest.mark.parametrize("method", [S.DARTS, S.PLAIN_UNIFORM_T])
def test_many_bins_without_shared_tiles(ctx, method):
    """A point sensor with 8192 bins: the warp tiles (warps x 3 x bins
    floats) no longer fit beside the table, so the launch commits with FP64
    atomics straight into the zeroed output.  Matched seeds against the
    oracle, histogram and sums of squares."""
    sc, sp = S.cube_workload(paths=1 << 17, seed=9)
    sc.gate.n_bins = 8192
    sp.method = method
    sp.max_bounces = 20
    hist, sq = ctx.render(sc, sp, sumsq=True)
    ctx.sync()
    h = hist.cpu().numpy()
    href, sqref, _ = O.render(sc, sp, method)
    assert np.count_nonzero(href) > 1500
    l2 = np.linalg.norm(h - href) / np.linalg.norm(href)
    assert l2 < 1e-3, l2
    if method == S.DARTS:
        # about 16 paths per bin: one path within its per-path allowance
        # moves its bin's square visibly, so the squares are compared in L2
        q = sq.cpu().numpy()
        assert np.linalg.norm(q - sqref) / np.linalg.norm(sqref) < 1e-3


def test_full_size_sampled_paths(ctx):
    """2^24 paths in the benchmark's launch configuration; 2048 sampled paths
    recomputed one by one by the oracle."""
    sc, sp = S.cube_workload(paths=1 << 24, seed=0)
    stride = (1 << 24) // 2048
    probe, pc, pb = ctx.probe(first=7, stride=stride, count=2048)
    ctx.render(sc, sp, probe=probe)
    ctx.sync()
    ids = 7 + stride * np.arange(2048)
    cdf = O.build_table(sc, sp)
    c_ref = np.zeros(2048)
    b_ref = np.zeros(2048, np.int64)
    flags = np.zeros(2048, np.int64)
    for i, pid in enumerate(ids):
        r = O.trace_paths(sc, sp, int(pid), 1, cdf=cdf)
        c_ref[i], b_ref[i], flags[i] = r["contrib"][0], r["bin"][0], r["flags"][0]
    assert np.array_equal(pb.cpu().numpy(), b_ref)
    gc = pc.cpu().numpy().astype(np.float64)
    rel = np.abs(gc - c_ref) / np.maximum(np.abs(c_ref), 1e-300)
    rel[(c_ref == 0) & (gc == 0)] = 0
    # paths whose trace flipped near a tie differ entirely; allow 1 %
    assert np.mean(rel > REL_PATH) <= 0.01, np.sort(rel)[-10:]
    st = ctx.stats()
    assert st["paths"] >= 1 << 24


def test_stats_match_oracle_counts(ctx):
    sc, sp = S.cube_workload(paths=1 << 15, seed=5)
    ctx.render(sc, sp)
    st = ctx.stats()
    _, _, ost = O.render(sc, sp, O.ORC_DARTS)
    assert abs(st["vertices"] - ost["vertices"]) <= 0.002 * ost["vertices"]
    assert abs(st["connections_nonempty"] - ost["connections_nonempty"]) <= 0.002 * ost["connections_nonempty"] + 5
    assert abs(st["escapes"] - ost["escapes"]) <= 0.002 * ost["escapes"] + 5


@pytest.mark.parametrize("method", [S.DARTS, S.PLAIN_UNIFORM_T])
def test_block_sizes_agree_and_autotune(ctx, method):
    """Every block size of the path kernel renders the same histogram (paths
    are assigned to blocks dynamically: equal up to FP64 summation order)."""
    sc, sp = S.cube_workload(paths=1 << 18, seed=21)
    sp.method = method
    outs = []
    for block in (512, 640, 768):
        ctx.set_launch(block)
        outs.append(ctx.render(sc, sp).cpu())
    ctx.set_launch(0)
    for o in outs[1:]:
        torch.testing.assert_close(o, outs[0], rtol=1e-6, atol=1e-15)
    href, _, _ = O.render(sc, sp, method)
    assert np.linalg.norm(outs[0].numpy() - href) <= 1e-3 * np.linalg.norm(href)
    best = ctx.autotune(sc, sp)
    assert best in (512, 640, 768)
    ctx.set_launch(0)
    from paper_2402_03106_gb300 import capi
    with pytest.raises(capi.DartsError):
        ctx.set_launch(100)


def test_launch_shapes_of_the_camera_kernel_agree(ctx):
    """The camera kernel of DARTS at 512, 640, 768 and 896 threads and with
    chunk caps from 1 to 1024 paths renders the same frame (the same paths
    with their FP64 atomics in another order), the lean kernel (camera in
    the medium, point emitters) and the general one (a zero-energy area
    emitter forces it); the autotuner keeps one of the shapes it timed;
    out-of-range shapes (896 for the batch kernel among them) are refused
    and change nothing."""
    sc = S.spheres_camera_scene(seed=0, width=64, height=64, n_bins=200)
    sp = S.Sampling(seed=4, paths_per_element=64, max_bounces=40)
    general = dataclasses.replace(sc, emitters=sc.emitters + [
        S.Emitter((2.0, 3.9, 2.0), 0.0, 0.0, S.EMITTER_AREA, (0.2, 0.0, 0.0), (0.0, 0.0, 0.2))])
    for scene in (sc, general):
        ref = None
        for block, chunk in ((512, 0), (640, 0), (768, 0), (896, 0), (512, 1), (640, 7), (768, 1024), (896, 128)):
            ctx.set_launch_config(block=block, chunk=chunk)
            h = ctx.render(scene, sp).cpu()
            if ref is None:
                ref = h
            else:
                torch.testing.assert_close(h, ref, rtol=1e-9, atol=1e-15)
    ctx.set_launch_config()
    best = ctx.autotune(sc, sp)
    cfg = ctx.launch_config()
    assert best in (512, 640, 768, 896) and cfg["block"] == best and cfg["chunk"] in (16, 32, 64, 128, 256)
    from paper_2402_03106_gb300 import capi
    for bad in (dict(block=100), dict(chunk=-1), dict(chunk=2000), dict(batch_items=65), dict(batch_block=1),
                dict(batch_block=896)):
        with pytest.raises(capi.DartsError):
            ctx.set_launch_config(**bad)
    assert ctx.launch_config() == cfg
    ctx.set_launch_config()


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
def test_empty_render_writes_zeros(ctx):
    sc, sp = S.cube_workload(paths=0)
    h = ctx.render(sc, sp)
    ctx.sync()
    assert torch.all(h == 0)


@pytest.mark.parametrize("n", [1, 255, 256 * 3 + 77])
def test_ragged_path_counts(ctx, n):
    sc, sp = S.cube_workload(paths=n, seed=11)
    h = ctx.render(sc, sp).cpu().numpy()
    ctx.sync()
    href, _, _ = O.render(sc, sp, O.ORC_DARTS)
    assert np.array_equal(h != 0, href != 0) or np.linalg.norm(h - href) <= 1e-3 * np.linalg.norm(href)
    np.testing.assert_allclose(h, href, rtol=1e-3, atol=1e-6 * max(href.max(), 1e-30))


def test_gate_before_straight_line_time_is_zero(ctx):
    sc = S.slab_scene(n_bins=4, t_min=0.2, t_max=0.7)
    for m in (S.DARTS, S.PLAIN_UNIFORM_T, S.VANILLA_DIRECT):
        sp = S.Sampling(seed=0, paths_per_element=4096, method=m)
        h = ctx.render(sc, sp)
        ctx.sync()
        assert torch.all(h == 0)
    st = ctx.stats()
    assert st["vertices"] > 0


def test_render_host_matches_device(ctx):
    sc, sp = S.cube_workload(paths=1 << 14, seed=3)
    h_dev = ctx.render(sc, sp).cpu()
    ctx.sync()
    hh = torch.zeros(256, dtype=torch.float64).pin_memory()
    ctx.render_host(sc, sp, hh)
    # path-to-block assignment is dynamic: equal up to FP64 summation order
    torch.testing.assert_close(hh, h_dev, rtol=1e-6, atol=1e-15)
    # the prepared form, with a sum of squares and a path offset (camera frame)
    sc2, sp2 = S.box_camera_workload(seed=1)
    sp2.paths_per_element = 2
    pr = ctx.prepare(sc2, sp2)
    d_h, d_q = ctx.render(sc2, sp2, sumsq=True, path_offset=4096 * 2)
    hh2 = torch.zeros(S.histogram_shape(sc2), dtype=torch.float64).pin_memory()
    hq2 = torch.zeros_like(hh2).pin_memory()
    pr.render_host(hh2, hq2, path_offset=4096 * 2)
    torch.testing.assert_close(hh2, d_h.cpu(), rtol=1e-6, atol=1e-15)
    torch.testing.assert_close(hq2, d_q.cpu(), rtol=1e-6, atol=1e-15)
    assert float(hh2.sum()) > 0.0


def test_render_host_async_pipeline(ctx):
    """Queued host renders: four frames in a row into four pinned buffers
    (the copy of each overlapping the next render, two device histograms
    alternating), then a larger scene (the device buffers grow); after
    sync every buffer equals the device render of its path range."""
    sc, sp = S.box_camera_workload(seed=2)
    sp.paths_per_element = 4
    n = S.total_paths(sc, sp)
    shape = S.histogram_shape(sc)
    pr = ctx.prepare(sc, sp)
    hs = [torch.zeros(shape, dtype=torch.float64).pin_memory() for _ in range(4)]
    qs = [torch.zeros(shape, dtype=torch.float64).pin_memory() for _ in range(4)]
    for i in range(4):
        pr.render_host_async(hs[i], qs[i] if i % 2 else None, path_offset=i * n)
    big = S.box_camera_scene(seed=2, width=96, height=64)
    hb = torch.zeros(S.histogram_shape(big), dtype=torch.float64).pin_memory()
    ctx.render_host_async(big, sp, hb)
    ctx.sync()
    for i in range(4):
        ref, refq = ctx.render(sc, sp, sumsq=True, path_offset=i * n)
        torch.testing.assert_close(hs[i], ref.cpu(), rtol=1e-6, atol=1e-15)
        if i % 2:
            torch.testing.assert_close(qs[i], refq.cpu(), rtol=1e-6, atol=1e-15)
    torch.testing.assert_close(hb, ctx.render(big, sp).cpu(), rtol=1e-6, atol=1e-15)
    assert float(hs[3].sum()) > 0.0


@pytest.mark.parametrize("kind", ["point", "camera"])
def test_accumulate_adds_into_the_outputs(ctx, kind):
    """DARTS_FLAG_ACCUMULATE: a second render of the next path range adds its
    estimate (and squares) into the first one's buffers -- the block-partial
    reduction of a point sensor and the atomics of a camera alike -- and the
    host-buffer, batched and adjoint calls refuse the flag."""
    import copy
    from paper_2402_03106_gb300 import capi
    if kind == "point":
        sc, sp = S.cube_workload(paths=1 << 14, seed=4)
    else:
        sc, sp = S.box_camera_workload(seed=4)
        sp.paths_per_element = 2
    n = S.total_paths(sc, sp)
    a, qa = ctx.render(sc, sp, sumsq=True)
    b, qb = ctx.render(sc, sp, sumsq=True, path_offset=n)
    acc = copy.deepcopy(sp)
    acc.flags |= S.FLAG_ACCUMULATE
    h, q = a.clone(), qa.clone()
    ctx.prepare(sc, acc).render(out=h, sumsq=q, path_offset=n)
    ctx.sync()
    torch.testing.assert_close(h, a + b, rtol=1e-9, atol=1e-300)
    torch.testing.assert_close(q, qa + qb, rtol=1e-9, atol=1e-300)
    assert float(b.abs().sum()) > 0.0
    hh = torch.zeros(S.histogram_shape(sc), dtype=torch.float64).pin_memory()
    for call in (lambda: ctx.render_host(sc, acc, hh),
                 lambda: ctx.adjoint(sc, acc, torch.ones(h.numel(), dtype=torch.float64))):
        with pytest.raises(capi.DartsError) as ei:
            call()
        assert ei.value.status == 6


def test_progressive_render_resumes_from_a_checkpoint(ctx):
    """Checkpoint / resume of a progressive render: Philox is keyed by the
    global path id, so a render is the sum of renders of consecutive path
    ranges.  Two ranges accumulate, the histogram and the next path offset
    are saved to the host, a new context restores them and accumulates two
    more; the result equals the uninterrupted run of four ranges in one
    context (up to FP64 summation order)."""
    from paper_2402_03106_gb300 import capi
    sc, sp = S.box_camera_workload(seed=6)
    sp.paths_per_element = 2
    n = S.total_paths(sc, sp)
    acc = S.Sampling(**{**sp.__dict__, "flags": sp.flags | S.FLAG_ACCUMULATE})
    h = torch.zeros(S.histogram_shape(sc), dtype=torch.float64, device="cuda")
    pr = ctx.prepare(sc, acc)
    for k in range(2):
        pr.render(out=h, path_offset=k * n)
    ctx.sync()
    saved, next_offset = h.cpu(), 2 * n  # the checkpoint
    del h
    ctx2 = capi.Context(0)
    try:
        h2 = saved.cuda()
        pr2 = ctx2.prepare(sc, acc)
        for k in range(2):
            pr2.render(out=h2, path_offset=next_offset + k * n)
        ctx2.sync()
        ref = torch.zeros_like(h2)
        pr3 = ctx2.prepare(sc, acc)
        for k in range(4):
            pr3.render(out=ref, path_offset=k * n)
        ctx2.sync()
        torch.testing.assert_close(h2, ref, rtol=1e-9, atol=1e-300)
        assert float(ref.sum()) > 0.0
    finally:
        ctx2.close()


def test_allocation_failure_is_reported(ctx):
    """A host render whose histogram cannot be allocated on the device (a
    2^15 x 2^15 camera x 4096 bins: 32 TB) returns DARTS_ERR_OOM before
    anything is launched, and the context stays usable.  A camera beyond
    2^30 pixels is refused outright."""
    from paper_2402_03106_gb300 import capi
    hh = torch.zeros(1, dtype=torch.float64)
    sc = S.box_camera_scene(seed=0, width=1 << 15, height=1 << 15, n_bins=4096)
    with pytest.raises(capi.DartsError) as ei:
        capi.darts_render_host(ctx.h, sc, S.Sampling(paths_per_element=1), hh, None, 0)
    assert ei.value.status == 3
    sc = S.box_camera_scene(seed=0, width=1 << 16, height=1 << 15, n_bins=1)
    with pytest.raises(capi.DartsError) as ei:
        capi.darts_render_host(ctx.h, sc, S.Sampling(paths_per_element=1), hh, None, 0)
    assert ei.value.status == 1
    small, sp = S.cube_workload(paths=1 << 10, seed=1)
    h = ctx.render(small, sp)
    ctx.sync()
    assert float(h.sum()) > 0.0


def test_other_ris_m_and_table_dims(ctx):
    sc, _ = S.cube_workload()
    sp = S.Sampling(seed=8, paths_per_element=1 << 12, ris_m=5, table_n_rho=7, table_n_s=5,
                    table_n_mu=100, max_bounces=10)
    gpu = ctx.debug_paths(sc, sp, 0, 1024)
    ref = O.trace_paths(sc, sp, 0, 1024)
    check_paths(gpu, ref, 10)


def test_invalid_arguments_are_rejected(ctx):
    from paper_2402_03106_gb300 import capi
    sc, sp = S.cube_workload(paths=16)
    bad = [
        ("sigma", lambda s, p: setattr(s.medium, "sigma_s", 0.0) or setattr(s.medium, "sigma_a", 0.0)),
        ("g", lambda s, p: setattr(s.medium, "g", 1.0)),
        ("bins", lambda s, p: setattr(s.gate, "n_bins", 0)),
        ("gate", lambda s, p: setattr(s.gate, "t_max", s.gate.t_min)),
        ("K", lambda s, p: setattr(p, "max_bounces", 0)),
        ("M", lambda s, p: setattr(p, "ris_m", 33)),
        ("alpha", lambda s, p: setattr(p, "mis_alpha", 0.0)),
        ("emitter", lambda s, p: setattr(s.emitters[0], "pos", (2.0, 0.5, 0.5))),
        ("method", lambda s, p: setattr(p, "method", 7)),
    ]
    import copy
    for name, mut in bad:
        s2, p2 = copy.deepcopy(sc), copy.deepcopy(sp)
        mut(s2, p2)
        with pytest.raises(capi.DartsError) as ei:
            ctx.render(s2, p2)
        assert ei.value.status == 1, name
    s2 = copy.deepcopy(sc)
    s2.emitters = s2.emitters * 9  # at most 8 emitters
    with pytest.raises(capi.DartsError) as ei:
        ctx.render(s2, sp)
    assert ei.value.status == 6
    ctx.sync()


def test_non_finite_contributions_are_reported(ctx):
    """Failure detection without a fault: an emitter energy beyond FP32
    range makes every contribution infinite.  The kernels drop them, set the
    device status word, and darts_sync reports DARTS_ERR_NUMERIC once; the
    next render is clean.  Point sensor (specialised kernel) and camera
    (general kernel)."""
    import copy
    from paper_2402_03106_gb300 import capi
    cube, sp = S.cube_workload(paths=1 << 12, seed=1)
    cam = S.box_camera_scene(seed=0, width=8, height=8, n_bins=64)
    for sc, spp in ((cube, sp.paths_per_element), (cam, 8)):
        hot = copy.deepcopy(sc)
        hot.emitters[0].energy = 1e40  # finite in FP64, infinite in FP32
        sp2 = S.Sampling(seed=3, paths_per_element=spp, max_bounces=10)
        h = ctx.render(hot, sp2)
        with pytest.raises(capi.DartsError) as ei:
            ctx.sync()
        assert ei.value.status == 4
        assert torch.isfinite(h).all()
        h = ctx.render(sc, sp2)
        ctx.sync()
        assert torch.isfinite(h).all() and float(h.sum()) > 0.0


# ---------------------------------------------------------------------------
# Physics on the GPU (statistical)
# ---------------------------------------------------------------------------
def test_gpu_single_scatter_closed_form(ctx):
    sc = S.infinite_scene(1.0, 0.01, 0.7, separation=1.0, n_bins=12, t_min=1.02, t_max=3.0)
    ref = O.single_scatter_bins(sc)
    n = 1 << 22
    sp = S.Sampling(seed=11, paths_per_element=n, max_bounces=1)
    for m in (S.DARTS, S.PLAIN_UNIFORM_T):
        sp.method = m
        h, sq = ctx.render(sc, sp, sumsq=True)
        ctx.sync()
        h, sq = h.cpu().numpy(), sq.cpu().numpy()
        se = O.standard_error(h, sq, n / 12 if m == S.DARTS else n)
        z = (h - ref) / se
        assert np.max(np.abs(z)) < 5.0, (m, z)


def test_gpu_darts_agrees_with_plain_pt(ctx):
    sc, _ = S.cube_workload()
    n = 1 << 22
    hd, sd = ctx.render(sc, S.Sampling(seed=1, paths_per_element=n), sumsq=True)
    hp, spq = ctx.render(sc, S.Sampling(seed=2, paths_per_element=n, method=S.PLAIN_UNIFORM_T), sumsq=True)
    ctx.sync()
    hd, sd, hp, spq = (t.cpu().numpy() for t in (hd, sd, hp, spq))
    se = np.sqrt(O.standard_error(hd, sd, n / 256) ** 2 + O.standard_error(hp, spq, n) ** 2)
    z = (hd - hp) / np.maximum(se, 1e-300)
    good = se > 0
    assert np.median(np.abs(z[1:][good[1:]])) < 1.5
    assert np.mean(np.abs(z[1:][good[1:]]) > 4) < 0.02
