"""Batched persistent launch of many media (darts_render_batch)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_03106_gb300 import scenes as S  # noqa: E402

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


def _media(n, seed=0, lo=10.0, hi=15.0):
    return S.batched_media(n_media=n, seed=seed, log2_budget=(lo, hi))


def test_batch_equals_single_renders(ctx):
    media = _media(24, seed=3)
    scenes = [m[0] for m in media]
    samplings = [m[1] for m in media]
    outs = ctx.render_batch(scenes, samplings)
    ctx.sync()
    st = ctx.stats()
    assert st["paths"] == sum(sp.paths_per_element for sp in samplings)
    for sc, sp, h in zip(scenes, samplings, outs):
        ref = ctx.render(sc, sp)
        torch.testing.assert_close(h, ref, rtol=1e-5, atol=1e-14 * float(ref.abs().max()) + 1e-300)


def test_tuned_batch_equals_single_renders(ctx):
    """darts_autotune_batch times every batch block size and item
    granularity, keeps the fastest on the context, and the batch in that
    shape (and in the extreme shapes) still equals the single renders."""
    media = _media(24, seed=7)
    scenes = [m[0] for m in media]
    samplings = [m[1] for m in media]
    outs = [torch.empty(sc.gate.n_bins, dtype=torch.float64, device="cuda") for sc in scenes]
    cfg = ctx.autotune_batch(scenes, samplings, outs)
    assert cfg["batch_block"] in (512, 640, 768) and cfg["batch_items"] in (2, 4, 8, 16, 32)
    refs = [ctx.render(sc, sp) for sc, sp in zip(scenes, samplings)]
    for shape in (cfg, dict(batch_block=512, batch_items=1), dict(batch_block=768, batch_items=64)):
        ctx.set_launch_config(batch_block=shape["batch_block"], batch_items=shape["batch_items"])
        got = ctx.render_batch(scenes, samplings)
        ctx.sync()
        for h, ref in zip(got, refs):
            torch.testing.assert_close(h, ref, rtol=1e-5, atol=1e-14 * float(ref.abs().max()) + 1e-300)
    ctx.set_launch_config()


def test_full_size_batch_equals_single_renders(ctx):
    """The batched configuration at full size: 256 media, budgets
    2^U[12,20] (about 47 M paths), 128 bins, in the benchmark's launch (one
    graph-captured persistent kernel); each medium's histogram equals its
    single render up to FP64 summation order.  The single renders are
    checked against the oracle elsewhere."""
    media = S.batched_media(n_media=256, seed=0)
    scenes = [m[0] for m in media]
    samplings = [m[1] for m in media]
    outs = ctx.render_batch(scenes, samplings)
    ctx.sync()
    st = ctx.stats()
    assert st["paths"] == sum(sp.paths_per_element for sp in samplings) > 40_000_000
    for sc, sp, h in zip(scenes, samplings, outs):
        ref = ctx.render(sc, sp)
        torch.testing.assert_close(h, ref, rtol=1e-5, atol=1e-14 * float(ref.abs().max()) + 1e-300)


def test_batch_matches_oracle(ctx):
    media = _media(4, seed=5, lo=12.0, hi=13.0)
    scenes = [m[0] for m in media]
    samplings = [dataclasses.replace(m[1], max_bounces=20) for m in media]
    outs = ctx.render_batch(scenes, samplings)
    ctx.sync()
    for sc, sp, h in zip(scenes, samplings, outs):
        href, sq, _ = O.render(sc, sp, O.ORC_DARTS)
        se = O.standard_error(href, sq, sp.paths_per_element / sc.gate.n_bins)
        hh = h.cpu().numpy()
        assert np.linalg.norm(hh - href) <= 1e-3 * np.linalg.norm(href) + 1e-300
        assert np.all(np.abs(hh - href) <= 3 * se + 1e-12 * np.abs(href).max())


def test_batch_graph_replay_recapture_and_direct(ctx):
    media = _media(8, seed=9)
    scenes = [m[0] for m in media]
    samplings = [m[1] for m in media]
    a = [t.clone() for t in ctx.render_batch(scenes, samplings)]
    outs = ctx.render_batch(scenes, samplings)  # replay of the cached graph
    for x, y in zip(a, outs):
        torch.testing.assert_close(x, y, rtol=1e-6, atol=1e-300)
    direct = ctx.render_batch(scenes, samplings, graph=False)
    for x, y in zip(a, direct):
        torch.testing.assert_close(x, y, rtol=1e-6, atol=1e-300)
    scenes2 = list(scenes)
    scenes2[3] = dataclasses.replace(scenes[3], medium=dataclasses.replace(scenes[3].medium, sigma_s=2.5))
    b = ctx.render_batch(scenes2, samplings)  # changed argument: re-captured
    ref = ctx.render(scenes2[3], samplings[3])
    torch.testing.assert_close(b[3], ref, rtol=1e-5, atol=1e-300)
    ctx.sync()


def test_batch_rejects_mixed_tables(ctx):
    from paper_2402_03106_gb300 import capi
    media = _media(2, seed=1)
    scenes = [m[0] for m in media]
    samplings = [m[1] for m in media]
    samplings[1] = dataclasses.replace(samplings[1], table_n_mu=128)
    with pytest.raises(capi.DartsError) as ei:
        ctx.render_batch(scenes, samplings)
    assert ei.value.status == 6
