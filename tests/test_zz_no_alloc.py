"""darts_render_static: rendering without a context and without device
allocation.

Callers that may not call cudaMalloc -- a plug-in whose host application owns
all device memory, a pipeline that must not allocate after start-up -- cannot
create a darts context (it allocates scratch).  This entry point takes its
scratch from a fixed device array inside the library instead.  The test calls
it through the C ABI and compares it with the context-based darts_render on
two calls in a row (the second call must not see the first call's counters),
then checks that oversized requests are refused.  It lives in a file of its
own that sorts last, and it needs no state from other tests.
"""
import copy

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_static_render_matches_context_render_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi, scenes as S

    sc, sp = S.cube_workload(paths=1 << 18, seed=13)
    ctx = capi.Context(0)
    ref_h, ref_q = ctx.render(sc, sp, sumsq=True)
    ctx.sync()
    for call in range(2):
        h = torch.full((sc.gate.n_bins,), float("nan"), dtype=torch.float64, device="cuda")
        q = torch.full_like(h, float("nan"))
        capi.darts_render_static(sc, sp, h, q)
        torch.cuda.synchronize()
        # same kernels and the same paths; only the FP64 summation order of the
        # block partials may differ (paths are handed to blocks dynamically)
        torch.testing.assert_close(h, ref_h, rtol=1e-6, atol=1e-15)
        torch.testing.assert_close(q, ref_q, rtol=1e-6, atol=1e-15)
    ctx.close()


def test_static_render_of_a_camera_and_of_many_bins():
    """A camera frame, and a point sensor whose 4096 bins are too many for the
    shared-memory tiles, add straight into the zeroed outputs: they need no
    block partials, so the static render takes them and matches darts_render."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi, scenes as S

    ctx = capi.Context(0)
    scc = S.box_camera_scene(seed=0, width=32, height=24, n_bins=128)
    spc = S.Sampling(seed=5, paths_per_element=16, max_bounces=20)
    big, spb = S.cube_workload(paths=1 << 16, seed=2)
    big.gate.n_bins = 4096
    for sc, sp in ((scc, spc), (big, spb)):
        ref_h, ref_q = ctx.render(sc, sp, sumsq=True)
        ctx.sync()
        for call in range(2):
            h = torch.full_like(ref_h, float("nan"))
            q = torch.full_like(ref_h, float("nan"))
            capi.darts_render_static(sc, sp, h, q)
            torch.cuda.synchronize()
            # FP64 atomics from dynamically scheduled paths: summation order only
            torch.testing.assert_close(h, ref_h, rtol=1e-9, atol=1e-15)
            torch.testing.assert_close(q, ref_q, rtol=1e-9, atol=1e-15)
    ctx.close()


def test_static_render_refuses_sizes_beyond_its_scratch():
    """A refused request is checked before anything is enqueued: the outputs
    keep their contents, and a following render is unaffected."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2402_03106_gb300 import capi, scenes as S

    sc, sp = S.cube_workload(paths=1024, seed=1)
    sp_big = copy.deepcopy(sp)
    sp_big.table_n_rho, sp_big.table_n_s = 64, 8  # 512 rows x 260 floats > 65536
    h = torch.full((sc.gate.n_bins,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.DartsError) as ei:
        capi.darts_render_static(sc, sp_big, h)
    assert ei.value.status == 6
    torch.cuda.synchronize()
    assert bool((h == 7.0).all()), "a refused call touched its output"
    capi.darts_render_static(sc, sp, h)
    ctx = capi.Context(0)
    ref = ctx.render(sc, sp)
    ctx.sync()
    torch.cuda.synchronize()
    torch.testing.assert_close(h, ref, rtol=1e-6, atol=1e-15)
    ctx.close()
