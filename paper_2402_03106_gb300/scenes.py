"""Scene and sampling descriptions, plus the seeded synthetic workloads.

This module holds plain numbers only: it performs none of the method's
arithmetic, so both the CUDA library binding and the CPU oracle used by the
tests can take their inputs from it.

The quantities follow the statement of the problem in the DARTS paper
(He et al. 2024): a homogeneous medium (sigma_s, sigma_a, Henyey-Greenstein g,
speed of light v = c/eta inside the medium, Eq. 3 and Eq. 9), pulse emitters
with start times (Eq. 1, t_e), a sensor, a time gate split into equal bins,
a path budget and a seed.  Lengths and times share units with v = 1
(Eq. 3 treats path length and time as interchangeable).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Methods (values are the ones of the C-ABI enum darts_method).
DARTS = 0
PLAIN_UNIFORM_T = 1
VANILLA_DIRECT = 2
DARTS_FULL_GATE = 3  # DARTS samplers over the whole gate, each connection binned by its time
METHOD_NAMES = {DARTS: "darts", PLAIN_UNIFORM_T: "plain_uniform_t", VANILLA_DIRECT: "vanilla_direct",
                DARTS_FULL_GATE: "darts_full_gate"}

# Sampling flags (C-ABI DARTS_FLAG_*).
FLAG_SENSOR_UNIFORM_ONLY = 1 << 0
FLAG_REBUILD_TABLE = 1 << 1
FLAG_NO_DA_DISTANCE = 1 << 2  # ablation: truncated-exponential distances (no DA target)
FLAG_NO_EDA = 1 << 3          # ablation: phase-function directions only (gamma = 0)
FLAG_IID_CANDIDATES = 1 << 4  # RIS candidates from independent uniforms (not the Sobol row)
FLAG_EQUIANGULAR = 1 << 5     # RIS candidates from the equiangular density about the emitter
FLAG_RESERVOIR = 1 << 6       # RIS selection by weighted reservoir sampling
FLAG_ACCUMULATE = 1 << 7      # darts_render adds into its outputs instead of overwriting them
FLAG_SURFACE_EDA = 1 << 8     # EDA / cosine-lobe MIS directions at surface vertices

Vec3 = Tuple[float, float, float]


@dataclass
class Medium:
    sigma_s: float
    sigma_a: float
    g: float
    v: float = 1.0


EMITTER_POINT = 0
EMITTER_AREA = 1
SENSOR_POINT = 0
SENSOR_PINHOLE = 1


@dataclass
class Emitter:
    """Pulse emitter: an isotropic point (kind 0), or a one-sided Lambertian
    parallelogram pos + s u + t v emitting toward u x v (kind 1)."""
    pos: Vec3
    t0: float = 0.0
    energy: float = 1.0
    kind: int = EMITTER_POINT
    u: Vec3 = (0.0, 0.0, 0.0)
    v: Vec3 = (0.0, 0.0, 0.0)


@dataclass
class Sensor:
    """Isotropic point fluence detector (kind 0, one element) or a pinhole
    camera at pos (kind 1, width x height elements, vertical FOV)."""
    pos: Vec3
    kind: int = SENSOR_POINT
    look_at: Vec3 = (0.0, 0.0, 1.0)
    up: Vec3 = (0.0, 1.0, 0.0)
    fov_deg: float = 40.0
    width: int = 1
    height: int = 1

    @property
    def elements(self) -> int:
        return self.width * self.height if self.kind == SENSOR_PINHOLE else 1


@dataclass
class Gate:
    """Time gate [t_min, t_max) in n_bins equal bins.  weights (optional):
    the sensor's temporal response W, one value >= 0 per bin; DARTS then
    samples each path's target bin from W (zero-weight bins get no paths)
    and the W-weighted pixel value is sum_b W_b h_b."""
    t_min: float
    t_max: float
    n_bins: int
    weights: Optional[Sequence[float]] = None


# Box faces that carry walls: bit 2*axis + side (side 1 = the high face).
WALL_X_LO, WALL_X_HI, WALL_Y_LO, WALL_Y_HI, WALL_Z_LO, WALL_Z_HI = (1 << i for i in range(6))


@dataclass
class Geometry:
    """Axis-aligned medium box [lo, hi]; optional opaque Lambertian walls on
    some faces and opaque Lambertian spheres (cx, cy, cz, r, albedo)."""
    lo: Vec3 = (0.0, 0.0, 0.0)
    hi: Vec3 = (1.0, 1.0, 1.0)
    walls: int = 0
    wall_albedo: float = 0.0
    spheres: List[Tuple[float, float, float, float, float]] = field(default_factory=list)


@dataclass
class Scene:
    medium: Medium
    geometry: Geometry
    emitters: List[Emitter]
    sensor: Sensor
    gate: Gate


@dataclass
class Sampling:
    seed: int = 0
    paths_per_element: int = 1 << 16
    max_bounces: int = 50
    ris_m: int = 8
    table_n_rho: int = 16
    table_n_s: int = 8
    table_n_mu: int = 256
    mis_alpha: float = 0.5
    method: int = DARTS
    flags: int = 0
    stream: int = 0


def slab_scene(sigma_s=1.0, sigma_a=0.01, g=0.7, v=1.0, side=1.0, n_bins=256,
               t_min=0.8, t_max=6.0) -> Scene:
    """The medium-only cube of side `side` with emitter and sensor on its axis.

    Emitter at (0.5, 0.5, 0.1)*side, t0 = 0, unit energy; point sensor at
    (0.5, 0.5, 0.9)*side; gate [t_min, t_max)*side split into n_bins bins.
    side = 1 with the defaults is the 2^16-path parity workload.
    """
    s = float(side)
    return Scene(
        medium=Medium(sigma_s, sigma_a, g, v),
        geometry=Geometry((0.0, 0.0, 0.0), (s, s, s)),
        emitters=[Emitter((0.5 * s, 0.5 * s, 0.1 * s), 0.0, 1.0)],
        sensor=Sensor((0.5 * s, 0.5 * s, 0.9 * s)),
        gate=Gate(t_min * s, t_max * s, n_bins),
    )


def cube_workload(paths: int = 1 << 16, seed: int = 0) -> Tuple[Scene, Sampling]:
    """Unit cube, sigma_s = 1, sigma_a = 0.01, g = 0.7, 256 bins on [0.8, 6),
    `paths` paths from `seed`, 50 bounces, 8 RIS candidates, 16x8x256 table."""
    return slab_scene(), Sampling(seed=seed, paths_per_element=paths)


def infinite_scene(sigma_s, sigma_a, g, separation=1.0, n_bins=64, t_min=None,
                   t_max=None, half_width=1.0e4) -> Scene:
    """Emitter and sensor `separation` apart inside a box so large that no
    path reaches its walls within the gate (an infinite medium in practice)."""
    c = separation
    t_min = c if t_min is None else t_min
    t_max = 6.0 * c if t_max is None else t_max
    h = float(half_width)
    return Scene(
        medium=Medium(sigma_s, sigma_a, g, 1.0),
        geometry=Geometry((-h, -h, -h), (h, h, h)),
        emitters=[Emitter((0.0, 0.0, 0.0), 0.0, 1.0)],
        sensor=Sensor((0.0, 0.0, float(c))),
        gate=Gate(float(t_min), float(t_max), n_bins),
    )


def box_camera_scene(seed: int = 0, width: int = 64, height: int = 64, n_bins: int = 512,
                     t_max: float = 16.0) -> Scene:
    """2x2x2 box with five Lambertian walls (albedo 0.5; the front face z = 0
    is open) filled with a medium drawn from the seed (sigma_s U[0.5, 2],
    albedo U[0.9, 0.99], g U[0, 0.9]); a 0.3 x 0.3 Lambertian pulse emitter
    centred on the ceiling (1, 2, 1) facing -y; a pinhole camera at
    (1, 1, -2.5) looking +z through the open face, 40 degree FOV."""
    rs = np.random.default_rng(np.random.SeedSequence([seed, 0xB0C5]))
    sigma_s = float(rs.uniform(0.5, 2.0))
    albedo = float(rs.uniform(0.9, 0.99))
    g = float(rs.uniform(0.0, 0.9))
    sigma_a = sigma_s * (1.0 - albedo) / albedo
    walls = WALL_X_LO | WALL_X_HI | WALL_Y_LO | WALL_Y_HI | WALL_Z_HI
    return Scene(
        medium=Medium(sigma_s, sigma_a, g, 1.0),
        geometry=Geometry((0.0, 0.0, 0.0), (2.0, 2.0, 2.0), walls, 0.5, []),
        emitters=[Emitter((0.85, 2.0, 0.85), 0.0, 1.0, EMITTER_AREA, (0.3, 0.0, 0.0), (0.0, 0.0, 0.3))],
        sensor=Sensor((1.0, 1.0, -2.5), SENSOR_PINHOLE, (1.0, 1.0, 0.0), (0.0, 1.0, 0.0), 40.0,
                      width, height),
        gate=Gate(0.0, t_max, n_bins),
    )


def box_camera_workload(seed: int = 0) -> Tuple[Scene, Sampling]:
    """64 x 64 pinhole view of the walled box, 16 paths per pixel, 512 bins."""
    return box_camera_scene(seed), Sampling(seed=seed, paths_per_element=16, max_bounces=50)


def cube_camera_scene(width: int = 32, height: int = 32) -> Scene:
    """The unit-cube medium seen by a 32 x 32 pinhole camera at
    (0.5, 0.5, -1.5) looking +z (40 degree FOV); 256 bins on [0.8, 6) shifted
    by the 1.5 camera leg."""
    sc = slab_scene()
    sc.sensor = Sensor((0.5, 0.5, -1.5), SENSOR_PINHOLE, (0.5, 0.5, 0.0), (0.0, 1.0, 0.0), 40.0,
                       width, height)
    sc.gate = Gate(0.8 + 1.5, 6.0 + 1.5, 256)
    return sc


def spheres_camera_scene(seed: int = 0, width: int = 512, height: int = 512, n_spheres: int = 32,
                         n_bins: int = 1000) -> Scene:
    """4x4x4 medium (sigma_s 0.8, sigma_a 0.005, g 0.8) with seeded opaque
    Lambertian spheres (radius U[0.05, 0.3], albedo U[0.2, 0.8]), two point
    pulse emitters at (1, 3.5, 1) t0 = 0 and (3, 3.5, 3) t0 = 1.5, a pinhole
    camera inside at (2, 2, 0.05) looking +z; 1000 bins on [0, 20)."""
    rs = np.random.default_rng(np.random.SeedSequence([seed, 0x5FE5]))
    emitters = [Emitter((1.0, 3.5, 1.0), 0.0, 1.0), Emitter((3.0, 3.5, 3.0), 1.5, 1.0)]
    cam = (2.0, 2.0, 0.05)
    spheres = []
    while len(spheres) < n_spheres:
        r = float(rs.uniform(0.05, 0.3))
        c = rs.uniform(r, 4.0 - r, size=3)
        keep = all(np.linalg.norm(c - np.array(p)) > r + 1e-3 for p in [e.pos for e in emitters] + [cam])
        alb = float(rs.uniform(0.2, 0.8))
        if keep:
            spheres.append((float(c[0]), float(c[1]), float(c[2]), r, alb))
    return Scene(
        medium=Medium(0.8, 0.005, 0.8, 1.0),
        geometry=Geometry((0.0, 0.0, 0.0), (4.0, 4.0, 4.0), 0, 0.0, spheres),
        emitters=emitters,
        sensor=Sensor(cam, SENSOR_PINHOLE, (2.0, 2.0, 1.0), (0.0, 1.0, 0.0), 40.0, width, height),
        gate=Gate(0.0, 20.0, n_bins),
    )


def batched_media(n_media: int = 256, seed: int = 0, n_bins: int = 128,
                  log2_budget: Tuple[float, float] = (12.0, 20.0)) -> List[Tuple[Scene, Sampling]]:
    """Independent slab media with uneven path budgets.

    Per medium: sigma_s log-uniform in [0.1, 10], albedo uniform in
    [0.5, 0.999], g uniform in [-0.3, 0.9], cube side uniform in [0.5, 4],
    path budget 2^U[12, 20] rounded to an integer; 128 bins.
    """
    rs = np.random.default_rng(np.random.SeedSequence([seed, 0x0D47]))
    out = []
    for i in range(n_media):
        sigma_s = float(10.0 ** rs.uniform(-1.0, 1.0))
        albedo = float(rs.uniform(0.5, 0.999))
        g = float(rs.uniform(-0.3, 0.9))
        side = float(rs.uniform(0.5, 4.0))
        budget = int(round(2.0 ** rs.uniform(*log2_budget)))
        sigma_a = sigma_s * (1.0 - albedo) / albedo
        sc = slab_scene(sigma_s, sigma_a, g, 1.0, side, n_bins)
        sp = Sampling(seed=seed, paths_per_element=budget, stream=i)
        out.append((sc, sp))
    return out


def with_paths(sp: Sampling, n: int) -> Sampling:
    return replace(sp, paths_per_element=int(n))


def total_paths(sc: Scene, sp: Sampling) -> int:
    """Number of paths one render call traces (every sensor element)."""
    return int(sp.paths_per_element) * sc.sensor.elements


def histogram_shape(sc: Scene) -> Tuple[int, ...]:
    """Shape of a render's output: [n_bins] for a point sensor,
    [height, width, n_bins] for a pinhole camera."""
    if sc.sensor.kind == SENSOR_PINHOLE:
        return (int(sc.sensor.height), int(sc.sensor.width), int(sc.gate.n_bins))
    return (int(sc.gate.n_bins),)
