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


def test_static_render_refuses_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2402_03106_gb300 import capi, scenes as S

    sc, sp = S.cube_workload(paths=1024, seed=1)
    big = copy.deepcopy(sc)
    big.gate.n_bins = 4096
    h = torch.zeros(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.DartsError) as ei:
        capi.darts_render_static(big, sp, h)
    assert ei.value.status == 6
    sp_big = copy.deepcopy(sp)
    sp_big.table_n_rho, sp_big.table_n_s = 64, 8  # 512 rows x 260 floats > 65536
    with pytest.raises(capi.DartsError) as ei:
        capi.darts_render_static(sc, sp_big, h[: sc.gate.n_bins])
    assert ei.value.status == 6
