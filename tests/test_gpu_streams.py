"""Contexts on separate CUDA streams share no state: frames rendered with
two or three in flight (one context per stream, frame i on stream i mod n)
equal the same frames rendered one after another on a single context.  The
camera frame sums FP64 atomics in arrival order, so the comparison allows
FP64 rounding; the point sensor's tiles are compared the same way."""
import pytest

torch = pytest.importorskip("torch")

from paper_2402_03106_gb300 import scenes as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi as c
    return c


def _workloads():
    cam, spc = S.box_camera_workload(seed=1)
    spc.paths_per_element = 4
    spc.flags |= S.FLAG_REBUILD_TABLE
    cube, spq = S.cube_workload(paths=1 << 16, seed=1)
    return [("camera", cam, spc), ("cube", cube, spq)]


@pytest.mark.parametrize("n_streams", [2, 3])
@pytest.mark.parametrize("which", [0, 1])
def test_frames_in_flight_equal_sequential_frames(capi, n_streams, which):
    name, sc, sp = _workloads()[which]
    N = S.total_paths(sc, sp)
    frames = 6
    ref_ctx = capi.Context(0)
    ref = [ref_ctx.render(sc, sp, path_offset=i * N).clone() for i in range(frames)]
    ref_ctx.sync()
    ref_ctx.close()
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    ctxs = [capi.Context(0, st) for st in streams]
    preps = [c.prepare(sc, sp) for c in ctxs]
    outs = [torch.full(S.histogram_shape(sc), float("nan"), dtype=torch.float64, device="cuda")
            for _ in range(frames)]
    torch.cuda.synchronize()  # the fills ran on the current stream, the renders do not
    for i in range(frames):  # queued back to back: the streams overlap on the device
        preps[i % n_streams].render(out=outs[i], path_offset=i * N)
    for c in ctxs:
        c.sync()
        c.close()
    torch.cuda.synchronize()
    for i in range(frames):
        a, b = outs[i], ref[i]
        assert torch.isfinite(a).all(), (name, i)
        scale = float(b.abs().max())
        assert scale > 0.0, (name, i)
        torch.testing.assert_close(a, b, rtol=1e-9, atol=1e-12 * scale, msg=f"{name} frame {i}")
    # different frames are different path ids: they must not coincide
    assert not torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("in_flight", [1, 2, 4])
@pytest.mark.parametrize("which", [0, 1])
def test_render_frames_equals_sequential_frames(capi, in_flight, which):
    """darts_render_frames: frame i holds what darts_render writes at path
    offset path_offset + i*N, sums of squares included; work enqueued on the
    context's stream after the call sees every frame complete."""
    name, sc, sp = _workloads()[which]
    N = S.total_paths(sc, sp)
    frames, off = 5, 3 * N
    ctx = capi.Context(0)
    ref = [ctx.render(sc, sp, sumsq=True, path_offset=off + i * N) for i in range(frames)]
    ref = [(h.clone(), q.clone()) for h, q in ref]
    outs, sqs = ctx.render_frames(sc, sp, frames, path_offset=off, in_flight=in_flight, sumsq=True)
    totals = torch.stack([o.sum() for o in outs])  # on the context's stream, no synchronisation
    ctx.sync()
    for i in range(frames):
        for a, b, what in ((outs[i], ref[i][0], "hist"), (sqs[i], ref[i][1], "sumsq")):
            scale = float(b.abs().max())
            assert scale > 0.0, (name, i, what)
            torch.testing.assert_close(a, b, rtol=1e-9, atol=1e-12 * scale, msg=f"{name} frame {i} {what}")
    torch.testing.assert_close(totals, torch.stack([r[0].sum() for r in ref]), rtol=1e-9, atol=0.0)
    ctx.close()


def test_render_frames_arguments_and_lane_status(capi):
    """Invalid arguments are refused before any launch; a non-finite frame
    on a lane is reported by the parent's darts_sync, once."""
    import copy
    sc, sp = S.cube_workload(paths=1 << 12, seed=4)
    ctx = capi.Context(0)
    prep = ctx.prepare(sc, sp)
    outs = [torch.empty(S.histogram_shape(sc), dtype=torch.float64, device="cuda") for _ in range(3)]
    for bad in (0, 5):
        with pytest.raises(capi.DartsError) as ei:
            prep.render_frames(outs, in_flight=bad)
        assert ei.value.status == 1
    with pytest.raises(capi.DartsError) as ei:
        prep.render_frames([])
    assert ei.value.status == 1
    acc = copy.deepcopy(sp)
    acc.flags |= S.FLAG_ACCUMULATE
    with pytest.raises(capi.DartsError) as ei:
        ctx.prepare(sc, acc).render_frames(outs)
    assert ei.value.status == 6
    hot = copy.deepcopy(sc)
    hot.emitters[0].energy = 1e40  # finite in FP64, infinite in FP32
    ctx.prepare(hot, sp).render_frames(outs, in_flight=3)
    with pytest.raises(capi.DartsError) as ei:
        ctx.sync()
    assert ei.value.status == 4
    prep.render_frames(outs, in_flight=3)
    ctx.sync()
    assert all(torch.isfinite(o).all() and float(o.sum()) > 0.0 for o in outs)
    ctx.close()
