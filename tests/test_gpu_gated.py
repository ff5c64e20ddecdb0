"""GPU parity for time-gated rendering with a temporal response W (Eq. 1-4;
Sec. 5.2 samples each DARTS path's target interval from W; Fig. 7 counts
the samples a zero weight rejects).

Tolerances as in test_gpu_parity: the bin of every path bit-exact (the
systematic sampling of W is decided in FP64 by the same arithmetic on both
sides), decision traces identical up to near-tie flips, contributions to
1e-4 (widened by the window conditioning), histograms within relative L2
1e-3 at matched seeds, and sample / rejection counts within 0.5 %.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_03106_gb300 import scenes as S  # noqa: E402
from parity_util import check_paths, displaced_sensitivity  # noqa: E402

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


def two_peak(n_bins, t_min, t_max, peaks):
    t = t_min + (np.arange(n_bins) + 0.5) * (t_max - t_min) / n_bins
    w = np.zeros(n_bins)
    for c, s_ in peaks:
        w += np.exp(-0.5 * ((t - c) / s_) ** 2)
    w[w < 1e-3] = 0.0
    return [float(x) for x in w]


def cube_w():
    # gate edges off the table's cell edges (C/S_M and S_M / S_max not round)
    sc = S.slab_scene(1.0, 0.02, 0.5, n_bins=28, t_min=0.83, t_max=3.63)
    sc.gate.weights = two_peak(28, 0.83, 3.63, ((1.6, 0.12), (2.6, 0.2)))
    return sc


def box_w():
    sc = S.box_camera_scene(seed=0, width=8, height=8, n_bins=64, t_max=16.0)
    sc.gate.weights = two_peak(64, 0.0, 16.0, ((5.0, 0.4), (9.0, 0.6)))
    return sc


@pytest.mark.parametrize("name", ["cube", "box"])
def test_weighted_per_path_parity(ctx, name):
    sc = cube_w() if name == "cube" else box_w()
    spp = 1 << 13 if name == "cube" else 32
    sp = S.Sampling(seed=8, paths_per_element=spp, max_bounces=30)
    n = 2048
    gpu = ctx.debug_paths(sc, sp, 37, n)
    ref = O.trace_paths(sc, sp, 37, n)
    w = np.asarray(sc.gate.weights)
    assert np.all(w[ref["bin"] % sc.gate.n_bins] > 0)
    sens = 5.0 * displaced_sensitivity(sc, sp, 37, n, O.ORC_DARTS, ref) if name == "box" else None
    check_paths(gpu, ref, sp.max_bounces, extra_tol=sens)


@pytest.mark.parametrize("name", ["cube", "box"])
def test_weighted_histogram_parity(ctx, name):
    sc = cube_w() if name == "cube" else box_w()
    spp = 1 << 15 if name == "cube" else 64
    sp = S.Sampling(seed=9, paths_per_element=spp, max_bounces=20)
    h = ctx.render(sc, sp).cpu().numpy().reshape(-1)
    href, _, _ = O.render(sc, sp, O.ORC_DARTS)
    assert np.linalg.norm(h - href) <= 1e-3 * np.linalg.norm(href)
    w = np.tile(np.asarray(sc.gate.weights), h.size // sc.gate.n_bins)
    assert np.all(h[w == 0] == 0.0)


@pytest.mark.parametrize("method", [S.DARTS, S.PLAIN_UNIFORM_T, S.VANILLA_DIRECT])
@pytest.mark.parametrize("name", ["cube", "box"])
def test_sample_and_rejection_counts(ctx, name, method):
    sc = cube_w() if name == "cube" else box_w()
    spp = 1 << 14 if name == "cube" else 32
    sp = S.Sampling(seed=10, paths_per_element=spp, max_bounces=20, method=method)
    ctx.render(sc, sp)
    st = ctx.stats()
    _, _, ost = O.render(sc, sp, method)
    assert abs(st["samples"] - ost["samples"]) <= 0.005 * ost["samples"] + 5
    assert abs(st["rejected"] - ost["rejected"]) <= 0.005 * ost["samples"] + 5
    if method == S.DARTS and name == "cube":
        assert st["rejected"] == 0
    if method == S.VANILLA_DIRECT:
        assert st["rejected"] > 0.2 * st["samples"]


def test_weights_not_accepted_where_unsupported(ctx):
    from paper_2402_03106_gb300 import capi
    sc = cube_w()
    hist = torch.zeros(sc.gate.n_bins, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.DartsError) as ei:
        capi.darts_render_static(sc, S.Sampling(paths_per_element=64), hist)
    assert ei.value.status == 6
    with pytest.raises(capi.DartsError) as ei:
        ctx.render_batch([sc], [S.Sampling(paths_per_element=64)])
    assert ei.value.status == 6
    bad = cube_w()
    bad.gate.weights = [-1.0] + list(bad.gate.weights[1:])
    with pytest.raises(capi.DartsError) as ei:
        ctx.render(bad, S.Sampling(paths_per_element=64))
    assert ei.value.status == 1
    zero = cube_w()
    zero.gate.weights = [0.0] * zero.gate.n_bins
    with pytest.raises(capi.DartsError):
        ctx.render(zero, S.Sampling(paths_per_element=64))


def test_single_gate_time_gated_matches_oracle(ctx):
    """Time-gated rendering: one bin at a late time, the camera box."""
    sc = S.box_camera_scene(seed=0, width=8, height=8, n_bins=1, t_max=10.25)
    sc.gate.t_min = 10.0
    for method in (S.DARTS, S.PLAIN_UNIFORM_T, S.VANILLA_DIRECT):
        sp = S.Sampling(seed=12, paths_per_element=128, max_bounces=100, method=method)
        h = ctx.render(sc, sp).cpu().numpy().reshape(-1)
        href, _, _ = O.render(sc, sp, method)
        assert np.linalg.norm(h - href) <= 1e-3 * np.linalg.norm(href), method


def test_full_gate_counts_and_weights(ctx):
    """Full-gate DARTS under a temporal response: every sample lands in some
    bin; those in zero-weight bins are counted as rejected, as the oracle does."""
    sc = cube_w()
    sp = S.Sampling(seed=13, paths_per_element=1 << 14, max_bounces=20, method=S.DARTS_FULL_GATE)
    h = ctx.render(sc, sp).cpu().numpy()
    st = ctx.stats()
    href, _, ost = O.render(sc, sp, O.ORC_DARTS_FULL_GATE)
    assert np.linalg.norm(h - href) <= 1e-3 * np.linalg.norm(href)
    assert abs(st["samples"] - ost["samples"]) <= 0.005 * ost["samples"] + 5
    assert abs(st["rejected"] - ost["rejected"]) <= 0.005 * ost["samples"] + 5
    assert st["rejected"] > 0
