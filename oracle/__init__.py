"""FP64 CPU oracle for DARTS transient path tracing -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg and
reference arm of ``bench.py`` may import this package.  The CUDA library never reads, links
or calls it, and it never imports the CUDA library: the two share no code.
Inputs arrive as plain scene/sampling objects (attribute access only).

What lives here:
  * ctypes bindings of the C oracle (``darts_oracle.c``): Philox4x32-10,
    the transient DA Green's function (Eq. 9), HG, the ellipse geometry of
    Eq. 18/21 and the control-vertex density of Eq. 22, the elliptical DA
    direction table (Eq. 16-18), the step-by-step DARTS estimator
    (Eq. 5-22), the two baselines and the path-replay score.
  * closed forms used as pins (``single_scatter_bins``, ``da_bins``).

Parity status of each function (which pin fixes it) is listed in the
test module ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

ORC_DARTS, ORC_PLAIN_UNIFORM_T, ORC_VANILLA_DIRECT, ORC_DARTS_FULL_GATE = 0, 1, 2, 3
EV_NONE, EV_EARLY, EV_SCATTER, EV_ESCAPE, EV_INVALID, EV_MAXDEPTH = range(6)
FLAG_NEAR_DEGENERATE, FLAG_SMALL_TPRIME = 1, 2


class OrcEmitter(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("t0", C.c_double), ("energy", C.c_double),
                ("kind", C.c_int32), ("u", C.c_double * 3), ("v", C.c_double * 3)]


class OrcScene(C.Structure):
    _fields_ = [
        ("sigma_s", C.c_double), ("sigma_a", C.c_double), ("g", C.c_double), ("v", C.c_double),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("xe", C.c_double * 3), ("t0", C.c_double), ("energy", C.c_double),
        ("xs", C.c_double * 3),
        ("t_min", C.c_double), ("t_max", C.c_double), ("n_bins", C.c_int32),
        ("max_bounces", C.c_int32), ("ris_m", C.c_int32),
        ("n_rho", C.c_int32), ("n_s", C.c_int32), ("n_mu", C.c_int32),
        ("mis_alpha", C.c_double), ("seed", C.c_uint64), ("stream", C.c_uint32),
        ("sensor_uniform_only", C.c_int32), ("paths_per_element", C.c_uint64),
        ("ablation", C.c_int32),
        ("n_emitters", C.c_int32), ("em", OrcEmitter * 8),
        ("sensor_kind", C.c_int32), ("look_at", C.c_double * 3), ("up", C.c_double * 3),
        ("fov_deg", C.c_double), ("width", C.c_int32), ("height", C.c_int32),
        ("walls", C.c_int32), ("wall_albedo", C.c_double), ("n_spheres", C.c_int32),
        ("spheres", (C.c_double * 5) * 64),
        ("weights", C.POINTER(C.c_double)),
    ]


_lib = None


def load():
    """Build (if needed) and load liboracle.so."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    u32p = C.POINTER(C.c_uint32)
    lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.orc_u01.argtypes = [C.c_uint32]
    lib.orc_u01.restype = C.c_double
    lib.orc_log_phi.argtypes = [C.c_double] * 6
    lib.orc_log_phi.restype = C.c_double
    lib.orc_hg_pdf.argtypes = [C.c_double, C.c_double]
    lib.orc_hg_pdf.restype = C.c_double
    lib.orc_hg_sample.argtypes = [C.c_double, C.c_double]
    lib.orc_hg_sample.restype = C.c_double
    lib.orc_ellipse.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
    lib.orc_control_pdf.argtypes = [C.c_double] * 5
    lib.orc_control_pdf.restype = C.c_double
    lib.orc_gauss_legendre.argtypes = [C.c_int, dp, dp]
    lib.orc_radical_inverse2.argtypes = [C.c_uint32]
    lib.orc_radical_inverse2.restype = C.c_double
    sp = C.POINTER(OrcScene)
    lib.orc_build_table.argtypes = [sp, dp]
    lib.orc_build_table.restype = C.c_int
    lib.orc_table_bin_integral.argtypes = [sp, C.c_int, C.c_int, C.c_int]
    lib.orc_table_bin_integral.restype = C.c_double
    lib.orc_table_row.argtypes = [sp, C.c_double, C.c_double, dp]
    lib.orc_table_row.restype = C.c_int
    lib.orc_trace_paths.argtypes = [sp, C.c_int, dp, C.c_uint64, C.c_uint32, dp,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_uint8), dp,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32), dp, dp]
    lib.orc_trace_paths.restype = C.c_int
    lib.orc_render.argtypes = [sp, C.c_int, dp, C.c_uint64, C.c_uint64, C.c_int, dp, dp, dp]
    lib.orc_render.restype = C.c_int
    lib.orc_render_window.argtypes = [sp, C.c_int, dp, C.c_uint64, C.c_uint64, C.c_int, C.c_uint64,
                                      C.c_uint64, dp, dp, dp]
    lib.orc_render_window.restype = C.c_int
    lib.orc_ris_step.argtypes = [sp, C.c_uint64, C.c_int, dp, dp, C.c_double, C.c_double, dp, dp,
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32), dp]
    lib.orc_ris_step.restype = C.c_int
    lib.orc_trace_ray.argtypes = [sp, dp, dp, C.POINTER(C.c_int32), dp]
    lib.orc_trace_ray.restype = C.c_double
    lib.orc_camera_ray.argtypes = [sp, C.c_int32, C.c_double, C.c_double, dp, dp, dp]
    lib.orc_camera_ray.restype = C.c_int
    lib.orc_sample_emitter.argtypes = [sp, C.c_uint64, dp, dp]
    lib.orc_adjoint.argtypes = [sp, dp, C.c_uint64, C.c_uint64, C.c_int, dp, dp, dp]
    lib.orc_adjoint.restype = C.c_int
    _lib = lib
    return lib


def _ptr(a, ctype=C.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def make_scene(scene, sampling) -> OrcScene:
    """Flatten scene/sampling objects (attribute access only) into the C struct."""
    s = OrcScene()
    m = scene.medium
    s.sigma_s, s.sigma_a, s.g, s.v = m.sigma_s, m.sigma_a, m.g, m.v
    s.lo[:] = list(scene.geometry.lo)
    s.hi[:] = list(scene.geometry.hi)
    ems = scene.emitters
    if not 1 <= len(ems) <= 8:
        raise ValueError("the oracle models 1 to 8 emitters")
    e = ems[0]
    s.xe[:] = list(e.pos)
    s.t0 = min(x.t0 for x in ems)
    s.energy = e.energy
    s.n_emitters = len(ems)
    for i, x in enumerate(ems):
        s.em[i].pos[:] = list(x.pos)
        s.em[i].t0, s.em[i].energy = x.t0, x.energy
        s.em[i].kind = getattr(x, "kind", 0)
        s.em[i].u[:] = list(getattr(x, "u", (0.0, 0.0, 0.0)))
        s.em[i].v[:] = list(getattr(x, "v", (0.0, 0.0, 0.0)))
    sen = scene.sensor
    s.xs[:] = list(sen.pos)
    s.sensor_kind = getattr(sen, "kind", 0)
    s.look_at[:] = list(getattr(sen, "look_at", (0.0, 0.0, 1.0)))
    s.up[:] = list(getattr(sen, "up", (0.0, 1.0, 0.0)))
    s.fov_deg = getattr(sen, "fov_deg", 40.0)
    s.width, s.height = getattr(sen, "width", 1), getattr(sen, "height", 1)
    geo = scene.geometry
    s.walls = getattr(geo, "walls", 0)
    s.wall_albedo = getattr(geo, "wall_albedo", 0.0)
    sph = list(getattr(geo, "spheres", []))
    if len(sph) > 64:
        raise ValueError("at most 64 spheres")
    s.n_spheres = len(sph)
    for i, q in enumerate(sph):
        s.spheres[i][:] = [float(v) for v in q]
    s.t_min, s.t_max, s.n_bins = scene.gate.t_min, scene.gate.t_max, scene.gate.n_bins
    w = getattr(scene.gate, "weights", None)
    if w is not None:
        if len(w) != s.n_bins:
            raise ValueError("gate weights need one value per bin")
        s._weights = np.ascontiguousarray(w, dtype=np.float64)  # kept alive with the struct
        s.weights = s._weights.ctypes.data_as(C.POINTER(C.c_double))
    s.max_bounces, s.ris_m = sampling.max_bounces, sampling.ris_m
    s.n_rho, s.n_s, s.n_mu = sampling.table_n_rho, sampling.table_n_s, sampling.table_n_mu
    s.mis_alpha = sampling.mis_alpha
    s.seed = sampling.seed & 0xFFFFFFFFFFFFFFFF
    s.stream = sampling.stream & 0xFFFFFFFF
    s.sensor_uniform_only = 1 if (sampling.flags & 1) else 0
    s.paths_per_element = sampling.paths_per_element
    f = sampling.flags
    s.ablation = ((1 if f & (1 << 2) else 0) | (2 if f & (1 << 3) else 0) | (4 if f & (1 << 4) else 0)
                  | (8 if f & (1 << 5) else 0) | (16 if f & (1 << 6) else 0) | (32 if f & (1 << 8) else 0))
    return s


# ----------------------------------------------------------------------------
# Elementary functions
# ----------------------------------------------------------------------------
def philox(ctr, key):
    lib = load()
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def u01(x):
    return load().orc_u01(int(x) & 0xFFFFFFFF)


def log_phi(r, t, sigma_s, sigma_a, g, v=1.0):
    return load().orc_log_phi(r, t, sigma_s, sigma_a, g, v)


def hg_pdf(mu, g):
    return load().orc_hg_pdf(mu, g)


def hg_sample(g, xi):
    return load().orc_hg_sample(g, xi)


def ellipse(S, Cd, mu):
    t, r1 = C.c_double(), C.c_double()
    load().orc_ellipse(S, Cd, mu, C.byref(t), C.byref(r1))
    return t.value, r1.value


def control_pdf(pS, S, Cd, mu, r1):
    return load().orc_control_pdf(pS, S, Cd, mu, r1)


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    load().orc_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def radical_inverse2(i):
    return load().orc_radical_inverse2(i)


# ----------------------------------------------------------------------------
# Table, paths, histograms
# ----------------------------------------------------------------------------
_table_cache = {}


def build_table(scene, sampling) -> np.ndarray:
    """Direction table of the scene (cached per medium, S_max and dims: the
    table depends on nothing else).  Returns a copy."""
    s = make_scene(scene, sampling)
    key = (s.sigma_s, s.sigma_a, s.g, s.v, s.t_max - s.t0, s.n_rho, s.n_s, s.n_mu)  # t0 = earliest
    if key in _table_cache:
        return _table_cache[key].copy()
    rows = s.n_rho * s.n_s
    cdf = np.zeros((rows, s.n_mu + 1))
    rc = load().orc_build_table(C.byref(s), _ptr(cdf))
    if rc != 0:
        raise RuntimeError(f"orc_build_table failed ({rc})")
    if len(_table_cache) > 64:
        _table_cache.clear()
    _table_cache[key] = cdf
    return cdf.copy()


def table_bin_integral(scene, sampling, row, mu_bin, adaptive=False):
    s = make_scene(scene, sampling)
    return load().orc_table_bin_integral(C.byref(s), row, mu_bin, 1 if adaptive else 0)


def table_row(scene, sampling, Cd, SM):
    s = make_scene(scene, sampling)
    m = C.c_double()
    r = load().orc_table_row(C.byref(s), Cd, SM, C.byref(m))
    return r, m.value


def trace_paths(scene, sampling, first, count, method=ORC_DARTS, cdf=None):
    """Per-path records for path ids first..first+count-1."""
    s = make_scene(scene, sampling)
    if method in (ORC_DARTS, ORC_DARTS_FULL_GATE) and cdf is None:
        cdf = build_table(scene, sampling)
    K = s.max_bounces
    out = dict(
        contrib=np.zeros(count), bin=np.zeros(count, np.int32),
        decisions=np.zeros((count, K, 4), np.uint8), margin=np.zeros((count, K)),
        flags=np.zeros(count, np.int32), nvert=np.zeros(count, np.int32),
        cond=np.zeros(count), tabcond=np.zeros(count),
    )
    cdf_c = None if cdf is None else np.ascontiguousarray(cdf, dtype=np.float64)
    rc = load().orc_trace_paths(
        C.byref(s), method, _ptr(cdf_c), first, count, _ptr(out["contrib"]),
        _ptr(out["bin"], C.c_int32), _ptr(out["decisions"], C.c_uint8), _ptr(out["margin"]),
        _ptr(out["flags"], C.c_int32), _ptr(out["nvert"], C.c_int32), _ptr(out["cond"]),
        _ptr(out["tabcond"]))
    if rc != 0:
        raise ValueError(f"orc_trace_paths rejected the scene ({rc})")
    return out


def ris_step(scene, sampling, path_id, k, x, w, SM, dm):
    """Distance step of one vertex from an explicit state (test hook)."""
    s = make_scene(scene, sampling)
    M = s.ris_m
    d = np.zeros(M)
    lw = np.zeros(M)
    valid = np.zeros(M, np.int32)
    sel = C.c_int32()
    fac = C.c_double()
    xa = np.ascontiguousarray(x, np.float64)
    wa = np.ascontiguousarray(w, np.float64)
    r = load().orc_ris_step(C.byref(s), path_id, k, _ptr(xa), _ptr(wa), SM, dm, _ptr(d), _ptr(lw),
                            _ptr(valid, C.c_int32), C.byref(sel), C.byref(fac))
    return dict(status=r, d=d, logw=lw, valid=valid.astype(bool), sel=sel.value, factor=fac.value)


def trace_ray(scene, sampling, x, w):
    """Nearest surface along a ray from inside the box: (distance, kind, normal);
    kind 0 = open boundary, 1 = wall, 2 + i = sphere i."""
    s = make_scene(scene, sampling)
    k = C.c_int32()
    n = np.zeros(3)
    d = load().orc_trace_ray(C.byref(s), _ptr(np.ascontiguousarray(x, np.float64)),
                             _ptr(np.ascontiguousarray(w, np.float64)), C.byref(k), _ptr(n))
    return d, k.value, n


def camera_ray(scene, sampling, pixel, jx, jy):
    """(hit, entry point, direction, camera-leg length) of a pinhole ray."""
    s = make_scene(scene, sampling)
    x = np.zeros(3)
    w = np.zeros(3)
    leg = C.c_double()
    hit = load().orc_camera_ray(C.byref(s), pixel, jx, jy, _ptr(x), _ptr(w), C.byref(leg))
    return bool(hit), x, w, leg.value


def sample_emitter(scene, sampling, path_id, q):
    s = make_scene(scene, sampling)
    out = np.zeros(8)
    load().orc_sample_emitter(C.byref(s), path_id, _ptr(np.ascontiguousarray(q, np.float64)), _ptr(out))
    return dict(y=out[:3], n=out[3:6], wsel=out[6], intensity=out[7])


STAT_NAMES = ("paths", "vertices", "connections", "connections_nonempty", "ris_candidates",
              "early_exits", "all_invalid", "escapes", "samples", "rejected")


def render(scene, sampling, method=ORC_DARTS, n_paths=None, offset=0, threads=None, cdf=None,
           window=None):
    """Histogram [elements * n_bins] (time-integrated fluence per bin, unit
    energy; one row of n_bins per camera pixel), sum of squared per-path bin
    contributions, and event statistics.  n_paths defaults to every path of
    every element.  window = (first element, element count) keeps only those
    rows (every traced path must fall in them): a sample of a large frame
    without full-frame buffers."""
    s = make_scene(scene, sampling)
    elements = s.width * s.height if s.sensor_kind == 1 else 1
    n = sampling.paths_per_element * elements if n_paths is None else n_paths
    if method in (ORC_DARTS, ORC_DARTS_FULL_GATE) and cdf is None:
        cdf = build_table(scene, sampling)
    threads = threads or (os.cpu_count() or 1)
    rows = elements if window is None else int(window[1])
    hist = np.zeros(s.n_bins * rows)
    sumsq = np.zeros(s.n_bins * rows)
    stats = np.zeros(len(STAT_NAMES))
    cdf_c = None if cdf is None else np.ascontiguousarray(cdf, dtype=np.float64)
    if window is None:
        rc = load().orc_render(C.byref(s), method, _ptr(cdf_c), n, offset, threads, _ptr(hist),
                               _ptr(sumsq), _ptr(stats))
    else:
        rc = load().orc_render_window(C.byref(s), method, _ptr(cdf_c), n, offset, threads,
                                      int(window[0]), rows, _ptr(hist), _ptr(sumsq), _ptr(stats))
    if rc != 0:
        raise ValueError(f"orc_render rejected the scene or window ({rc})")
    return hist, sumsq, dict(zip(STAT_NAMES, stats.tolist()))


def standard_error(hist, sumsq, paths_per_bin):
    """Per-bin standard error from the sum of squared per-path contributions."""
    var = np.maximum(sumsq - hist * hist / np.maximum(paths_per_bin, 1), 0.0)
    return np.sqrt(var)


def adjoint(scene, sampling, dLdh, n_paths=None, offset=0, threads=None, cdf=None):
    """Path-replay gradient estimate of sum_b dLdh[b] * h_b w.r.t.
    (sigma_s, sigma_a, g), with per-path squared sums for a standard error."""
    s = make_scene(scene, sampling)
    elements = s.width * s.height if s.sensor_kind == 1 else 1
    n = sampling.paths_per_element * elements if n_paths is None else n_paths
    if cdf is None:
        cdf = build_table(scene, sampling)
    threads = threads or (os.cpu_count() or 1)
    g = np.zeros(3)
    gsq = np.zeros(3)
    d = np.ascontiguousarray(dLdh, dtype=np.float64)
    rc = load().orc_adjoint(C.byref(s), _ptr(np.ascontiguousarray(cdf, np.float64)), n, offset,
                            threads, _ptr(d), _ptr(g), _ptr(gsq))
    if rc != 0:
        raise ValueError(f"orc_adjoint rejected the scene ({rc})")
    return g, gsq


# ----------------------------------------------------------------------------
# Closed forms (pins)
# ----------------------------------------------------------------------------
def _hg_np(mu, g):
    den = 1.0 + g * g - 2.0 * g * mu
    return (1.0 - g * g) / (4.0 * math.pi * den * np.sqrt(den))


def single_scatter_rate(S, Cd, sigma_s, sigma_a, g, v=1.0, energy=1.0):
    """Fluence rate at time S/v from single scattering in an infinite medium.

    Derived from the ellipse geometry of Eq. 18 and the Jacobian of Eq. 22:
    phi_1 = v sigma_s I_e e^{-sigma_t S} * 2 pi * int_{-1}^{1} 2 f(cos theta_s)
    / (S^2 + C^2 - 2 S C mu) dmu, with I_e = E / 4 pi and
    cos theta_s = (C mu - t)/(S - t), t = (S^2 - C^2)/(2 (S - C mu)).
    For g = 0 it reduces to v sigma_s I_e e^{-sigma_t S} ln((S+C)/(S-C)) / (S C).
    """
    from scipy import integrate
    st = sigma_s + sigma_a
    Ie = energy / (4.0 * math.pi)
    if S <= Cd:
        return 0.0
    if g == 0.0:
        return v * sigma_s * Ie * math.exp(-st * S) * math.log((S + Cd) / (S - Cd)) / (S * Cd)

    def f(mu):
        t = (S * S - Cd * Cd) / (2.0 * (S - Cd * mu))
        r1 = S - t
        cs = (Cd * mu - t) / r1
        return 2.0 * _hg_np(cs, g) / (S * S + Cd * Cd - 2.0 * S * Cd * mu)

    val, _ = integrate.quad(f, -1.0, 1.0, limit=400, epsabs=0.0, epsrel=1e-11)
    return v * sigma_s * Ie * math.exp(-st * S) * 2.0 * math.pi * val


def single_scatter_bins(scene):
    """Time-integrated single-scatter fluence in each gate bin (infinite medium)."""
    from scipy import integrate
    m = scene.medium
    e = scene.emitters[0]
    Cd = float(np.linalg.norm(np.subtract(scene.sensor.pos, e.pos)))
    G = scene.gate
    dt = (G.t_max - G.t_min) / G.n_bins
    out = np.zeros(G.n_bins)
    for b in range(G.n_bins):
        S0 = m.v * (G.t_min + b * dt - e.t0)
        S1 = m.v * (G.t_min + (b + 1) * dt - e.t0)
        lo = max(S0, Cd)
        if S1 <= lo:
            continue
        val, _ = integrate.quad(
            lambda S: single_scatter_rate(S, Cd, m.sigma_s, m.sigma_a, m.g, m.v, e.energy),
            lo, S1, limit=400, epsabs=0.0, epsrel=1e-10)
        out[b] = val / m.v
    return out


def da_rate(r, t, sigma_s, sigma_a, g, v=1.0, energy=1.0):
    """Fluence rate of Eq. 9 at distance r and time t after the pulse."""
    return energy * math.exp(log_phi(r, t, sigma_s, sigma_a, g, v))


def da_bins(scene):
    """Eq. 9 integrated over each gate bin at the sensor position."""
    from scipy import integrate
    m = scene.medium
    e = scene.emitters[0]
    r = float(np.linalg.norm(np.subtract(scene.sensor.pos, e.pos)))
    G = scene.gate
    dt = (G.t_max - G.t_min) / G.n_bins
    out = np.zeros(G.n_bins)
    for b in range(G.n_bins):
        t0 = G.t_min + b * dt - e.t0
        t1 = t0 + dt
        val, _ = integrate.quad(lambda t: da_rate(r, t, m.sigma_s, m.sigma_a, m.g, m.v, e.energy),
                                max(t0, 1e-12), t1, limit=200)
        out[b] = val
    return out
