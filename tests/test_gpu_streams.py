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
