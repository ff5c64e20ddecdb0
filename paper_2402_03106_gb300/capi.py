"""Thin ctypes binding of libdarts (include/darts.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device memory and streams come from PyTorch.  The functions named
``darts_*`` mirror the C entry points one to one; ``Context`` and the
helpers below them allocate output tensors and convert the scene objects of
``scenes.py`` into the C structs.

The library is loaded from this package's directory; when it is missing the
import of this module still works but every call raises, so no path can
fall back silently to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import torch

from . import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdarts.so")
# the same library with every output, tile and table index checked on the
# device (DARTS_ERR_BOUNDS instead of an out-of-range access); load it with
# load(CHECKED_LIB_PATH) before the first context
CHECKED_LIB_PATH = os.path.join(HERE, "libdarts_checked.so")

DARTS_OK = 0
STATUS_NAMES = {0: "DARTS_OK", 1: "DARTS_ERR_INVALID_ARG", 2: "DARTS_ERR_CUDA", 3: "DARTS_ERR_OOM",
                4: "DARTS_ERR_NUMERIC", 5: "DARTS_ERR_TIMEOUT", 6: "DARTS_ERR_UNSUPPORTED",
                7: "DARTS_ERR_BOUNDS"}

EXPORTED = ("darts_create", "darts_destroy", "darts_set_stream", "darts_status_string",
            "darts_last_error", "darts_sync", "darts_build_table", "darts_table_row_stride",
            "darts_render", "darts_render_host", "darts_get_stats", "darts_debug_paths",
            "darts_debug_philox", "darts_set_kernel_timing", "darts_last_kernel_ms",
            "darts_render_static", "darts_set_launch", "darts_autotune", "darts_adjoint",
            "darts_render_batch", "darts_render_host_async", "darts_render_frames",
            "darts_load_table", "darts_set_launch_config", "darts_get_launch_config",
            "darts_autotune_batch")
BATCH_NO_GRAPH = 1


class DartsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class darts_medium(C.Structure):
    _fields_ = [("sigma_s", C.c_double), ("sigma_a", C.c_double), ("g", C.c_double), ("v", C.c_double)]


class darts_emitter(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("t0", C.c_double), ("energy", C.c_double),
                ("kind", C.c_int32), ("u", C.c_double * 3), ("v", C.c_double * 3)]


class darts_sensor(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("kind", C.c_int32), ("look_at", C.c_double * 3),
                ("up", C.c_double * 3), ("fov_deg", C.c_double), ("width", C.c_int32),
                ("height", C.c_int32)]


class darts_gate(C.Structure):
    _fields_ = [("t_min", C.c_double), ("t_max", C.c_double), ("n_bins", C.c_int32),
                ("weights", C.POINTER(C.c_double))]


class darts_geometry(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("walls", C.c_int32),
                ("wall_albedo", C.c_double), ("n_spheres", C.c_int32),
                ("spheres", C.POINTER(C.c_double))]


class darts_scene(C.Structure):
    _fields_ = [("medium", darts_medium), ("geom", darts_geometry),
                ("emitters", C.POINTER(darts_emitter)), ("n_emitters", C.c_int32),
                ("sensor", darts_sensor), ("gate", darts_gate)]


class darts_sampling(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("paths_per_element", C.c_uint64),
                ("max_bounces", C.c_int32), ("ris_m", C.c_int32),
                ("table_n_rho", C.c_int32), ("table_n_s", C.c_int32), ("table_n_mu", C.c_int32),
                ("mis_alpha", C.c_double), ("method", C.c_int32), ("flags", C.c_uint32),
                ("stream", C.c_uint32)]


class darts_probe(C.Structure):
    _fields_ = [("first", C.c_uint64), ("stride", C.c_uint64), ("count", C.c_uint32),
                ("contrib_dev", C.c_void_p), ("bin_dev", C.c_void_p)]


class darts_launch(C.Structure):
    _fields_ = [("block", C.c_int32), ("chunk", C.c_int32), ("batch_block", C.c_int32),
                ("batch_items", C.c_int32)]


class darts_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "paths", "vertices", "connections_nonempty", "distance_steps", "early_exits",
        "all_invalid", "escapes", "fp64_ellipse", "fp64_phi", "samples", "rejected")]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libdarts.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(path)
        vp, st = C.c_void_p, C.c_int
        sc_p, sp_p = C.POINTER(darts_scene), C.POINTER(darts_sampling)
        lib.darts_create.argtypes = [C.POINTER(vp), C.c_int, vp]
        lib.darts_destroy.argtypes = [vp]
        lib.darts_set_stream.argtypes = [vp, vp]
        lib.darts_status_string.argtypes = [st]
        lib.darts_status_string.restype = C.c_char_p
        lib.darts_last_error.argtypes = [vp, C.c_char_p, C.c_size_t]
        lib.darts_sync.argtypes = [vp]
        lib.darts_build_table.argtypes = [vp, sc_p, sp_p, vp]
        lib.darts_load_table.argtypes = [vp, sc_p, sp_p, vp]
        lib.darts_table_row_stride.argtypes = [C.c_int32]
        lib.darts_table_row_stride.restype = C.c_int32
        lib.darts_render.argtypes = [vp, sc_p, sp_p, vp, vp, C.c_uint64, C.POINTER(darts_probe)]
        lib.darts_render_host.argtypes = [vp, sc_p, sp_p, vp, vp, C.c_uint64]
        lib.darts_render_host_async.argtypes = [vp, sc_p, sp_p, vp, vp, C.c_uint64]
        lib.darts_render_frames.argtypes = [vp, sc_p, sp_p, C.c_uint32, vp, vp, C.c_uint64, C.c_int32]
        lib.darts_get_stats.argtypes = [vp, C.POINTER(darts_stats)]
        lib.darts_debug_paths.argtypes = [vp, sc_p, sp_p, C.c_uint64, C.c_uint32, vp, vp, vp, vp]
        lib.darts_debug_philox.argtypes = [vp, vp, C.c_uint64, C.c_uint32, vp]
        lib.darts_set_kernel_timing.argtypes = [vp, C.c_int]
        lib.darts_last_kernel_ms.argtypes = [vp, C.POINTER(C.c_float)]
        lib.darts_render_static.argtypes = [sc_p, sp_p, vp, vp, C.c_uint64, vp]
        lib.darts_set_launch.argtypes = [vp, C.c_int]
        lib.darts_adjoint.argtypes = [vp, sc_p, sp_p, vp, vp, vp, C.c_uint64]
        lib.darts_render_batch.argtypes = [vp, C.c_int, sc_p, sp_p, C.POINTER(C.c_void_p), C.c_uint32]
        lib.darts_autotune.argtypes = [vp, sc_p, sp_p, C.POINTER(C.c_int)]
        lib.darts_set_launch_config.argtypes = [vp, C.POINTER(darts_launch)]
        lib.darts_get_launch_config.argtypes = [vp, C.POINTER(darts_launch)]
        lib.darts_autotune_batch.argtypes = [vp, C.c_int, sc_p, sp_p, C.POINTER(C.c_void_p),
                                             C.POINTER(darts_launch)]
        for name in EXPORTED:
            if name not in ("darts_status_string", "darts_table_row_stride"):
                getattr(lib, name).restype = st
        _lib = lib
        return lib


# ----------------------------------------------------------------------------
# Scene conversion
# ----------------------------------------------------------------------------
def to_c_scene(scene: S.Scene):
    """Return (darts_scene, keepalive) for a scenes.Scene."""
    n = len(scene.emitters)
    arr = (darts_emitter * max(n, 1))()
    for i, e in enumerate(scene.emitters):
        arr[i].pos[:] = [float(x) for x in e.pos]
        arr[i].t0 = float(e.t0)
        arr[i].energy = float(e.energy)
        arr[i].kind = int(e.kind)
        arr[i].u[:] = [float(x) for x in e.u]
        arr[i].v[:] = [float(x) for x in e.v]
    cs = darts_scene()
    m = scene.medium
    cs.medium = darts_medium(float(m.sigma_s), float(m.sigma_a), float(m.g), float(m.v))
    geo = scene.geometry
    cs.geom.lo[:] = [float(x) for x in geo.lo]
    cs.geom.hi[:] = [float(x) for x in geo.hi]
    cs.geom.walls = int(geo.walls)
    cs.geom.wall_albedo = float(geo.wall_albedo)
    sph = (C.c_double * max(5 * len(geo.spheres), 1))()
    for k, q in enumerate(geo.spheres):
        sph[5 * k:5 * k + 5] = [float(x) for x in q]
    cs.geom.n_spheres = len(geo.spheres)
    cs.geom.spheres = C.cast(sph, C.POINTER(C.c_double))
    cs.emitters = C.cast(arr, C.POINTER(darts_emitter))
    cs.n_emitters = n
    sen = scene.sensor
    cs.sensor.pos[:] = [float(x) for x in sen.pos]
    cs.sensor.kind = int(sen.kind)
    cs.sensor.look_at[:] = [float(x) for x in sen.look_at]
    cs.sensor.up[:] = [float(x) for x in sen.up]
    cs.sensor.fov_deg = float(sen.fov_deg)
    cs.sensor.width = int(sen.width)
    cs.sensor.height = int(sen.height)
    cs.gate = darts_gate(float(scene.gate.t_min), float(scene.gate.t_max), int(scene.gate.n_bins))
    gw = getattr(scene.gate, "weights", None)
    wts = None
    if gw is not None:
        wts = (C.c_double * max(len(gw), 1))(*[float(x) for x in gw])
        cs.gate.weights = C.cast(wts, C.POINTER(C.c_double))
    return cs, (arr, sph, wts)


def to_c_sampling(sp: S.Sampling) -> darts_sampling:
    c = darts_sampling()
    c.seed = int(sp.seed) & 0xFFFFFFFFFFFFFFFF
    c.paths_per_element = int(sp.paths_per_element)
    c.max_bounces = int(sp.max_bounces)
    c.ris_m = int(sp.ris_m)
    c.table_n_rho, c.table_n_s, c.table_n_mu = int(sp.table_n_rho), int(sp.table_n_s), int(sp.table_n_mu)
    c.mis_alpha = float(sp.mis_alpha)
    c.method = int(sp.method)
    c.flags = int(sp.flags)
    c.stream = int(sp.stream) & 0xFFFFFFFF
    return c


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _ptr_array(ts: Optional[Sequence[torch.Tensor]]):
    """A C array of device pointers (double* const*), or None."""
    if ts is None:
        return None
    return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


# ----------------------------------------------------------------------------
# One-to-one wrappers of the C entry points
# ----------------------------------------------------------------------------
def _check(ctx_handle, status: int):
    if status != DARTS_OK:
        lib = load()
        msg = C.create_string_buffer(512)
        if ctx_handle:
            lib.darts_last_error(ctx_handle, msg, 512)
        raise DartsError(status, msg.value.decode() or lib.darts_status_string(status).decode())


def darts_create(device: int = 0, stream=None):
    h = C.c_void_p()
    _check(None, load().darts_create(C.byref(h), int(device), stream))
    return h


def darts_destroy(h):
    _check(None, load().darts_destroy(h))


def darts_set_stream(h, stream):
    _check(h, load().darts_set_stream(h, stream))


def darts_sync(h):
    _check(h, load().darts_sync(h))


def darts_table_row_stride(n_mu: int) -> int:
    return int(load().darts_table_row_stride(int(n_mu)))


def darts_build_table(h, scene, sampling, cdf: torch.Tensor):
    cs, keep = to_c_scene(scene)
    _check(h, load().darts_build_table(h, C.byref(cs), C.byref(to_c_sampling(sampling)), _ptr(cdf)))


def darts_load_table(h, scene, sampling, cdf: torch.Tensor):
    cs, keep = to_c_scene(scene)
    _check(h, load().darts_load_table(h, C.byref(cs), C.byref(to_c_sampling(sampling)), _ptr(cdf)))


def darts_render(h, scene, sampling, hist: torch.Tensor, sumsq: Optional[torch.Tensor] = None,
                 path_offset: int = 0, probe: Optional[darts_probe] = None):
    cs, keep = to_c_scene(scene)
    _check(h, load().darts_render(h, C.byref(cs), C.byref(to_c_sampling(sampling)), _ptr(hist),
                                  _ptr(sumsq), int(path_offset),
                                  C.byref(probe) if probe is not None else None))


def darts_render_host(h, scene, sampling, hist_host: torch.Tensor,
                      sumsq_host: Optional[torch.Tensor] = None, path_offset: int = 0):
    cs, keep = to_c_scene(scene)
    _check(h, load().darts_render_host(h, C.byref(cs), C.byref(to_c_sampling(sampling)),
                                       _ptr(hist_host), _ptr(sumsq_host), int(path_offset)))


def darts_get_stats(h) -> dict:
    st = darts_stats()
    _check(h, load().darts_get_stats(h, C.byref(st)))
    return {n: int(getattr(st, n)) for n, _ in darts_stats._fields_}


def darts_debug_paths(h, scene, sampling, first, count, contrib, bins, nvert, decisions):
    cs, keep = to_c_scene(scene)
    _check(h, load().darts_debug_paths(h, C.byref(cs), C.byref(to_c_sampling(sampling)),
                                       int(first), int(count), _ptr(contrib), _ptr(bins),
                                       _ptr(nvert), _ptr(decisions)))


def darts_debug_philox(h, ctr: torch.Tensor, seed: int, out: torch.Tensor):
    _check(h, load().darts_debug_philox(h, _ptr(ctr), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                        int(ctr.numel() // 4), _ptr(out)))


def darts_set_kernel_timing(h, enable: bool):
    _check(h, load().darts_set_kernel_timing(h, 1 if enable else 0))


def darts_last_kernel_ms(h) -> float:
    ms = C.c_float()
    _check(h, load().darts_last_kernel_ms(h, C.byref(ms)))
    return float(ms.value)


def darts_adjoint(h, scene, sampling, dLdh: torch.Tensor, grad3: torch.Tensor,
                  grad3_sq: Optional[torch.Tensor] = None, path_offset: int = 0):
    cs, keep = to_c_scene(scene)
    _check(h, load().darts_adjoint(h, C.byref(cs), C.byref(to_c_sampling(sampling)), _ptr(dLdh),
                                   _ptr(grad3), _ptr(grad3_sq), int(path_offset)))


def darts_render_batch(h, scenes, samplings, hists, flags: int = 0):
    n = len(scenes)
    cs_arr = (darts_scene * n)()
    keep = []
    for i, sc in enumerate(scenes):
        cs, k = to_c_scene(sc)
        cs_arr[i] = cs
        keep.append(k)
    sp_arr = (darts_sampling * n)(*[to_c_sampling(sp) for sp in samplings])
    ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in hists])
    _check(h, load().darts_render_batch(h, n, cs_arr, sp_arr, ptrs, int(flags)))


def _batch_arrays(scenes, samplings, hists):
    n = len(scenes)
    cs_arr = (darts_scene * n)()
    keep = []
    for i, sc in enumerate(scenes):
        cs, k = to_c_scene(sc)
        cs_arr[i] = cs
        keep.append(k)
    sp_arr = (darts_sampling * n)(*[to_c_sampling(sp) for sp in samplings])
    ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in hists])
    return cs_arr, sp_arr, ptrs, keep


def darts_autotune_batch(h, scenes, samplings, hists) -> dict:
    cs_arr, sp_arr, ptrs, keep = _batch_arrays(scenes, samplings, hists)
    out = darts_launch()
    _check(h, load().darts_autotune_batch(h, len(scenes), cs_arr, sp_arr, ptrs, C.byref(out)))
    return {f: int(getattr(out, f)) for f, _ in darts_launch._fields_}


def darts_set_launch_config(h, block: int = 0, chunk: int = 0, batch_block: int = 0, batch_items: int = 0):
    cfg = darts_launch(int(block), int(chunk), int(batch_block), int(batch_items))
    _check(h, load().darts_set_launch_config(h, C.byref(cfg)))


def darts_get_launch_config(h) -> dict:
    out = darts_launch()
    _check(h, load().darts_get_launch_config(h, C.byref(out)))
    return {f: int(getattr(out, f)) for f, _ in darts_launch._fields_}


def darts_set_launch(h, block: int):
    _check(h, load().darts_set_launch(h, int(block)))


def darts_autotune(h, scene, sampling) -> int:
    cs, keep = to_c_scene(scene)
    b = C.c_int()
    _check(h, load().darts_autotune(h, C.byref(cs), C.byref(to_c_sampling(sampling)), C.byref(b)))
    return int(b.value)


def darts_render_static(scene, sampling, hist: torch.Tensor, sumsq: Optional[torch.Tensor] = None,
                        path_offset: int = 0, stream=None):
    """darts_render_static: render without a context and without allocating
    device memory (for callers that may not call cudaMalloc); scratch comes
    from the library's fixed 4 MiB device array.  `stream` is a torch stream
    (default: the current stream of hist's device)."""
    cs, keep = to_c_scene(scene)
    if stream is None:
        stream = torch.cuda.current_stream(hist.device)
    _check(None, load().darts_render_static(C.byref(cs), C.byref(to_c_sampling(sampling)), _ptr(hist),
                                            _ptr(sumsq), int(path_offset),
                                            C.c_void_p(stream.cuda_stream)))


# ----------------------------------------------------------------------------
# Convenience layer
# ----------------------------------------------------------------------------
class Prepared:
    """A scene and sampling converted once into the C structs; render() then
    calls darts_render directly with them.  Changing the scene objects later
    does not affect a Prepared: prepare again."""

    def __init__(self, ctx: "Context", scene, sampling):
        self.ctx = ctx
        self.cs, self._keep = to_c_scene(scene)
        self.csp = to_c_sampling(sampling)
        self.shape = S.histogram_shape(scene)
        self._lib = load()

    def render(self, out: Optional[torch.Tensor] = None, sumsq: Optional[torch.Tensor] = None,
               path_offset: int = 0) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=self.ctx._dev())
        _check(self.ctx.h, self._lib.darts_render(self.ctx.h, C.byref(self.cs), C.byref(self.csp), _ptr(out),
                                                  _ptr(sumsq), int(path_offset), None))
        return out

    def render_host(self, hist_host: torch.Tensor, sumsq_host: Optional[torch.Tensor] = None,
                    path_offset: int = 0) -> torch.Tensor:
        """darts_render_host with the marshalled structs: host (pinned) buffers in
        and out, synchronised on return."""
        _check(self.ctx.h, self._lib.darts_render_host(self.ctx.h, C.byref(self.cs), C.byref(self.csp),
                                                       _ptr(hist_host), _ptr(sumsq_host), int(path_offset)))
        return hist_host

    def render_frames(self, outs: Sequence[torch.Tensor], sumsq: Optional[Sequence[torch.Tensor]] = None,
                      path_offset: int = 0, in_flight: int = 2) -> Sequence[torch.Tensor]:
        """darts_render_frames: frame i (path ids path_offset + i*N ...) into
        outs[i], up to in_flight frames running at once on the context's
        lanes; ordered on the context's stream like render()."""
        if sumsq is not None and len(sumsq) != len(outs):
            raise ValueError("one sumsq buffer per frame")
        _check(self.ctx.h, self._lib.darts_render_frames(self.ctx.h, C.byref(self.cs), C.byref(self.csp),
                                                         len(outs), _ptr_array(outs), _ptr_array(sumsq),
                                                         int(path_offset), int(in_flight)))
        return outs

    def render_host_async(self, hist_host: torch.Tensor, sumsq_host: Optional[torch.Tensor] = None,
                          path_offset: int = 0) -> torch.Tensor:
        """darts_render_host_async: queued render and copy back into pinned
        host buffers; the buffers are complete after Context.sync()."""
        _check(self.ctx.h, self._lib.darts_render_host_async(self.ctx.h, C.byref(self.cs), C.byref(self.csp),
                                                             _ptr(hist_host), _ptr(sumsq_host),
                                                             int(path_offset)))
        return hist_host

class Context:
    """A libdarts context on one CUDA device, ordered on a torch stream."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libdarts needs a CUDA device")
        self.device = int(device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.h = darts_create(self.device, C.c_void_p(self.stream.cuda_stream))

    def close(self):
        if self.h:
            darts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        darts_set_stream(self.h, C.c_void_p(stream.cuda_stream))

    def sync(self):
        darts_sync(self.h)

    def _dev(self):
        return torch.device("cuda", self.device)

    def render(self, scene, sampling, sumsq: bool = False, path_offset: int = 0,
               out: Optional[torch.Tensor] = None, probe: Optional[darts_probe] = None):
        shape = S.histogram_shape(scene)
        hist = out if out is not None else torch.empty(shape, dtype=torch.float64, device=self._dev())
        sq = torch.empty(shape, dtype=torch.float64, device=self._dev()) if sumsq else None
        darts_render(self.h, scene, sampling, hist, sq, path_offset, probe)
        return (hist, sq) if sumsq else hist

    def prepare(self, scene, sampling) -> "Prepared":
        """Marshal a scene and sampling once for repeated renders (the
        per-call conversion of render() costs tens of microseconds of host
        time, comparable to a whole camera frame on the GPU)."""
        return Prepared(self, scene, sampling)

    def render_host(self, scene, sampling, hist_host: torch.Tensor,
                    sumsq_host: Optional[torch.Tensor] = None, path_offset: int = 0):
        darts_render_host(self.h, scene, sampling, hist_host, sumsq_host, path_offset)
        return hist_host

    def render_host_async(self, scene, sampling, hist_host: torch.Tensor,
                          sumsq_host: Optional[torch.Tensor] = None, path_offset: int = 0):
        """Queued render into pinned host buffers (complete after sync())."""
        cs, keep = to_c_scene(scene)
        csp = to_c_sampling(sampling)
        _check(self.h, load().darts_render_host_async(self.h, C.byref(cs), C.byref(csp), _ptr(hist_host),
                                                      _ptr(sumsq_host), int(path_offset)))
        return hist_host

    def render_frames(self, scene, sampling, n_frames: int, path_offset: int = 0, in_flight: int = 2,
                      sumsq: bool = False):
        """n_frames frames of one scene (frame i: path ids path_offset + i*N
        ...), up to in_flight of them running at once; returns the list of
        histograms (and of sums of squares when sumsq)."""
        shape = S.histogram_shape(scene)
        outs = [torch.empty(shape, dtype=torch.float64, device=self._dev()) for _ in range(n_frames)]
        sqs = [torch.empty(shape, dtype=torch.float64, device=self._dev()) for _ in range(n_frames)] if sumsq else None
        self.prepare(scene, sampling).render_frames(outs, sqs, path_offset, in_flight)
        return (outs, sqs) if sumsq else outs

    def build_table(self, scene, sampling, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        rows = sampling.table_n_rho * sampling.table_n_s
        stride = darts_table_row_stride(sampling.table_n_mu)
        cdf = out if out is not None else torch.empty(rows, stride, dtype=torch.float32, device=self._dev())
        darts_build_table(self.h, scene, sampling, cdf)
        return cdf

    def load_table(self, scene, sampling, cdf: torch.Tensor):
        """Install a precomputed direction table (float32 [rows][row stride]
        on this context's device, the layout of build_table) as the cached
        table of the scene's medium; renders without FLAG_REBUILD_TABLE use it."""
        rows = sampling.table_n_rho * sampling.table_n_s
        stride = darts_table_row_stride(sampling.table_n_mu)
        if (cdf.dtype != torch.float32 or tuple(cdf.shape) != (rows, stride) or not cdf.is_contiguous()
                or cdf.device != self._dev()):
            raise ValueError(f"the table must be a contiguous float32 [{rows}][{stride}] tensor on {self._dev()}")
        darts_load_table(self.h, scene, sampling, cdf)

    def adjoint(self, scene, sampling, dLdh: torch.Tensor, sumsq: bool = False, path_offset: int = 0):
        """Gradient of sum_b dLdh[b] h_b w.r.t. (sigma_s, sigma_a, g) by path replay."""
        d = dLdh.to(device=self._dev(), dtype=torch.float64).contiguous()
        g3 = torch.empty(3, dtype=torch.float64, device=self._dev())
        q3 = torch.empty(3, dtype=torch.float64, device=self._dev()) if sumsq else None
        darts_adjoint(self.h, scene, sampling, d, g3, q3, path_offset)
        return (g3, q3) if sumsq else g3

    def render_batch(self, scenes, samplings, graph: bool = True, outs=None):
        """Histograms of many media from one persistent launch (CUDA graph)."""
        if outs is None:
            outs = [torch.empty(sc.gate.n_bins, dtype=torch.float64, device=self._dev()) for sc in scenes]
        darts_render_batch(self.h, scenes, samplings, outs, 0 if graph else BATCH_NO_GRAPH)
        return outs

    def set_launch(self, block: int):
        darts_set_launch(self.h, block)

    def autotune(self, scene, sampling) -> int:
        return darts_autotune(self.h, scene, sampling)

    def autotune_batch(self, scenes, samplings, outs) -> dict:
        """Tune the batched launch (block size, work items per CTA share) on
        these media; returns the context's launch shape."""
        return darts_autotune_batch(self.h, scenes, samplings, outs)

    def launch_config(self) -> dict:
        return darts_get_launch_config(self.h)

    def set_launch_config(self, block: int = 0, chunk: int = 0, batch_block: int = 0, batch_items: int = 0):
        darts_set_launch_config(self.h, block, chunk, batch_block, batch_items)

    def set_kernel_timing(self, enable: bool):
        darts_set_kernel_timing(self.h, enable)

    def last_kernel_ms(self) -> float:
        return darts_last_kernel_ms(self.h)

    def stats(self) -> dict:
        return darts_get_stats(self.h)

    def debug_paths(self, scene, sampling, first: int, count: int) -> dict:
        dev = self._dev()
        K = sampling.max_bounces
        out = dict(contrib=torch.zeros(count, dtype=torch.float32, device=dev),
                   bin=torch.zeros(count, dtype=torch.int32, device=dev),
                   nvert=torch.zeros(count, dtype=torch.int32, device=dev),
                   decisions=torch.zeros(count, K, 4, dtype=torch.uint8, device=dev))
        darts_debug_paths(self.h, scene, sampling, first, count, out["contrib"], out["bin"],
                          out["nvert"], out["decisions"])
        return out

    def probe(self, first: int, stride: int, count: int):
        dev = self._dev()
        c = torch.zeros(count, dtype=torch.float32, device=dev)
        b = torch.full((count,), -1, dtype=torch.int32, device=dev)
        p = darts_probe(int(first), int(stride), int(count), c.data_ptr(), b.data_ptr())
        return p, c, b

    def philox(self, ctr, seed: int) -> torch.Tensor:
        ctr = torch.as_tensor(ctr, dtype=torch.int64).reshape(-1).to(torch.uint32)
        ctr = ctr.to(self._dev())
        out = torch.zeros_like(ctr)
        darts_debug_philox(self.h, ctr, seed, out)
        return out
