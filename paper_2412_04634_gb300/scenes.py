"""Seeded synthetic inputs for the NIRC hot path.

This module only *produces data*: procedural scene descriptions (primitives,
camera), initial network parameters and the analytic training field of the
training-step workload.  It holds none of the method's arithmetic (no ray
tracing, no sampling, no encoding, no network evaluation), so both the CUDA
path and the CPU oracle can consume its output without sharing code.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64); the
method's own per-sample random numbers (Philox4x32-10) are generated inside
each implementation.

Binary layouts (little endian, 4-byte fields):

* scene blob  = 96-byte header + n_prims * 96-byte primitive records
* header      = u32 n_prims, u32 pad[3], f32 cam_origin[4], f32 cam_top_left[4],
                f32 cam_horizontal[4], f32 cam_vertical[4], u32 reserved[4]
* primitive   = f32 a[3], f32 radius, f32 u[3], f32 inv_uu, f32 v[3], f32 inv_vv,
                f32 n[3], u32 kind, f32 albedo[3], f32 roughness,
                f32 emission[3], u32 flags
  kind 0 = sphere (centre a, radius), kind 1 = rectangle (corner a, edges u, v
  with u . v = 0, unit normal n = u x v / |u x v|, inv_uu = 1/(u.u), inv_vv = 1/(v.v)).
  flags bits 0-1 = material (0 Lambertian, 1 Lambertian + GGX specular,
  2 black / non-scattering), bit 8 = emission on both sides (otherwise only
  on the side the stored normal points to).
* shading record (64 B) = f32 p[3], f32 n[3], f32 wo[3], f32 albedo[3],
  f32 roughness, u32 prim, u32 flags, u32 pad; flags bit 0 = valid,
  bits 1-2 = material.

Pixel (px, py) with jitter (jx, jy) looks along
cam_top_left + ((px+jx)/W) * cam_horizontal + ((py+jy)/H) * cam_vertical - cam_origin,
so pixel row 0 is the top of the image.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PRIM_DTYPE = np.dtype([
    ("a", "<f4", 3), ("radius", "<f4"),
    ("u", "<f4", 3), ("inv_uu", "<f4"),
    ("v", "<f4", 3), ("inv_vv", "<f4"),
    ("n", "<f4", 3), ("kind", "<u4"),
    ("albedo", "<f4", 3), ("roughness", "<f4"),
    ("emission", "<f4", 3), ("flags", "<u4"),
])
assert PRIM_DTYPE.itemsize == 96

HEADER_DTYPE = np.dtype([
    ("n_prims", "<u4"), ("pad", "<u4", 3),
    ("cam_origin", "<f4", 4), ("cam_top_left", "<f4", 4),
    ("cam_horizontal", "<f4", 4), ("cam_vertical", "<f4", 4),
    ("reserved", "<u4", 4),
])
assert HEADER_DTYPE.itemsize == 96

RECORD_DTYPE = np.dtype([
    ("p", "<f4", 3), ("n", "<f4", 3), ("wo", "<f4", 3), ("albedo", "<f4", 3),
    ("roughness", "<f4"), ("prim", "<u4"), ("flags", "<u4"), ("pad", "<u4"),
])
assert RECORD_DTYPE.itemsize == 64

KIND_SPHERE, KIND_RECT = 0, 1
MAT_LAMBERT, MAT_GGX, MAT_BLACK = 0, 1, 2
EMIT_TWO_SIDED = 1 << 8

EMITTER_RADIANCE = 10.0   # config "quad emitter of radiance 10"
EMITTER_SIZE = 0.1        # 0.1 x 0.1 quad
EMITTER_HEIGHT = 0.999    # just under the ceiling, facing -y


@dataclasses.dataclass
class Scene:
    """A scene blob plus the numpy views it was made from."""
    header: np.ndarray   # HEADER_DTYPE, shape ()
    prims: np.ndarray    # PRIM_DTYPE, shape (n,)
    width: int
    height: int
    emitter_phase: float = 0.0
    moving_emitter: bool = False
    env: np.ndarray | None = None  # cube-map texels, float32 (6 S S, 4); header reserved[0] = S

    def blob(self) -> np.ndarray:
        """Header, primitives and (if any) the environment cube map, as a uint8 array."""
        parts = [np.frombuffer(self.header.tobytes(), np.uint8), np.frombuffer(self.prims.tobytes(), np.uint8)]
        if self.env is not None:
            parts.append(np.frombuffer(np.ascontiguousarray(self.env, np.float32).tobytes(), np.uint8))
        return np.concatenate(parts)

    @property
    def n_prims(self) -> int:
        return int(self.prims.shape[0])


def _rect(corner, u, v):
    corner = np.asarray(corner, np.float64)
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    c = np.cross(u, v)
    n = c / np.linalg.norm(c)
    return corner, u, v, n


def _camera(origin, vfov_deg, width, height):
    """Pinhole camera looking along +z with image plane at distance 1."""
    origin = np.asarray(origin, np.float64)
    half_h = math.tan(math.radians(vfov_deg) / 2.0)
    half_w = half_h * (width / height)
    top_left = origin + np.array([-half_w, half_h, 1.0])
    horizontal = np.array([2.0 * half_w, 0.0, 0.0])
    vertical = np.array([0.0, -2.0 * half_h, 0.0])
    return origin, top_left, horizontal, vertical


def _header(n_prims, cam):
    h = np.zeros((), HEADER_DTYPE)
    h["n_prims"] = n_prims
    origin, top_left, horizontal, vertical = cam
    h["cam_origin"][:3] = origin
    h["cam_top_left"][:3] = top_left
    h["cam_horizontal"][:3] = horizontal
    h["cam_vertical"][:3] = vertical
    return h


def _fill_rect(p, corner, u, v, albedo, roughness, material, emission=(0, 0, 0), flags_extra=0):
    corner, u, v, n = _rect(corner, u, v)
    p["kind"] = KIND_RECT
    p["a"] = corner
    p["u"] = u
    p["v"] = v
    p["n"] = n
    p["inv_uu"] = 1.0 / float(np.dot(u, u))
    p["inv_vv"] = 1.0 / float(np.dot(v, v))
    p["radius"] = 0.0
    p["albedo"] = albedo
    p["roughness"] = roughness
    p["emission"] = emission
    p["flags"] = material | flags_extra


def _fill_sphere(p, centre, radius, albedo, roughness, material, emission=(0, 0, 0), flags_extra=0):
    p["kind"] = KIND_SPHERE
    p["a"] = centre
    p["radius"] = radius
    p["u"] = 0.0
    p["v"] = 0.0
    p["n"] = 0.0
    p["inv_uu"] = 0.0
    p["inv_vv"] = 0.0
    p["albedo"] = albedo
    p["roughness"] = roughness
    p["emission"] = emission
    p["flags"] = material | flags_extra


def emitter_centre(frame: int, phase: float, moving: bool):
    """Emitter centre: fixed at the ceiling centre, or moving on a circle of
    radius 0.25 around it with period 60 frames (the dynamic-scene workload)."""
    if not moving:
        return (0.5, EMITTER_HEIGHT, 0.5)
    ang = 2.0 * math.pi * frame / 60.0 + phase
    return (0.5 + 0.25 * math.cos(ang), EMITTER_HEIGHT, 0.5 + 0.25 * math.sin(ang))


def cornell_scene(width: int, height: int, seed: int = 1, n_prims: int = 8,
                  glossy: bool = False, frame: int = 0, moving_emitter: bool = False) -> Scene:
    """Procedural Cornell box.

    The box is the unit cube with an open front (z = 0): floor, ceiling, back
    wall and two side walls (5 rectangles), a 0.1 x 0.1 emitter of radiance 10
    just under the ceiling facing -y, then ``n_prims - 6`` random primitives.
    With ``n_prims == 8`` these are two spheres of radius U[0.1, 0.25]
    (the 64x64 correctness workload); larger counts mix small spheres and
    randomly oriented rectangles (the 1080p workload).  Albedos are
    U[0.2, 0.8] per channel; with ``glossy`` every non-emitter primitive uses
    the Lambertian + GGX material with roughness U[0.05, 1].
    """
    assert n_prims >= 6
    rng = np.random.default_rng(seed)
    prims = np.zeros(n_prims, PRIM_DTYPE)
    mat = MAT_GGX if glossy else MAT_LAMBERT

    def albedo():
        return rng.uniform(0.2, 0.8, 3)

    def rough():
        return float(rng.uniform(0.05, 1.0)) if glossy else 1.0

    walls = [
        ((0, 0, 0), (0, 0, 1), (1, 0, 0)),   # floor y = 0
        ((0, 1, 0), (1, 0, 0), (0, 0, 1)),   # ceiling y = 1
        ((0, 0, 1), (1, 0, 0), (0, 1, 0)),   # back wall z = 1
        ((0, 0, 0), (0, 1, 0), (0, 0, 1)),   # left wall x = 0
        ((1, 0, 0), (0, 0, 1), (0, 1, 0)),   # right wall x = 1
    ]
    for i, (c, u, v) in enumerate(walls):
        _fill_rect(prims[i], c, u, v, albedo(), rough(), mat)

    phase = float(rng.uniform(0.0, 2.0 * math.pi))
    cx, cy, cz = emitter_centre(frame, phase, moving_emitter)
    h = EMITTER_SIZE / 2.0
    # u x v = (0.1,0,0) x (0,0,0.1) points to -y: the emitting side faces the room.
    _fill_rect(prims[5], (cx - h, cy, cz - h), (EMITTER_SIZE, 0, 0), (0, 0, EMITTER_SIZE),
               (0, 0, 0), 1.0, MAT_BLACK, emission=(EMITTER_RADIANCE,) * 3)

    n_extra = n_prims - 6
    if n_prims == 8:
        for i in range(6, 8):
            r = float(rng.uniform(0.1, 0.25))
            c = rng.uniform(r, 1.0 - r, 3)
            c[1] = r + rng.uniform(0.0, 0.3)  # resting near the floor
            _fill_sphere(prims[i], c, r, albedo(), rough(), mat)
    else:
        for k in range(n_extra):
            i = 6 + k
            if k % 2 == 0:
                r = float(rng.uniform(0.02, 0.07))
                c = rng.uniform(0.05 + r, 0.95 - r, 3)
                _fill_sphere(prims[i], c, r, albedo(), rough(), mat)
            else:
                nrm = rng.normal(size=3)
                nrm /= np.linalg.norm(nrm)
                t = np.cross(nrm, [1.0, 0.0, 0.0] if abs(nrm[0]) < 0.9 else [0.0, 1.0, 0.0])
                t /= np.linalg.norm(t)
                b = np.cross(nrm, t)
                lu, lv = rng.uniform(0.04, 0.15, 2)
                centre = rng.uniform(0.1, 0.9, 3)
                u = t * lu
                v = b * lv
                corner = centre - 0.5 * u - 0.5 * v
                _fill_rect(prims[i], corner, u, v, albedo(), rough(), mat)

    cam = _camera((0.5, 0.5, -1.2), 40.0, width, height)
    sc = Scene(_header(n_prims, cam), prims, width, height)
    sc.emitter_phase = phase
    sc.moving_emitter = moving_emitter
    return sc


def scene_at_frame(scene: Scene, frame: int) -> Scene:
    """Copy of a Cornell scene with the emitter moved to its position at
    ``frame`` (the dynamic-scene workload); other primitives unchanged."""
    prims = scene.prims.copy()
    cx, cy, cz = emitter_centre(frame, scene.emitter_phase, scene.moving_emitter)
    h = EMITTER_SIZE / 2.0
    _fill_rect(prims[5], (cx - h, cy, cz - h), (EMITTER_SIZE, 0, 0), (0, 0, EMITTER_SIZE),
               (0, 0, 0), 1.0, MAT_BLACK, emission=(EMITTER_RADIANCE,) * 3)
    out = Scene(scene.header.copy(), prims, scene.width, scene.height)
    out.emitter_phase = scene.emitter_phase
    out.moving_emitter = scene.moving_emitter
    out.env = scene.env
    return out


def floor_light_scene(width: int, height: int, rho: float = 0.5, emission: float = 4.0,
                      glossy: bool = False, roughness: float = 0.3) -> Scene:
    """A unit floor (y = 0, normal +y, albedo ``rho``) under a 0.3 x 0.3
    emitter at height 0.5 facing -y; the camera looks at the floor from
    above.  Direct light on the floor has a closed form (the irradiance of a
    polygonal emitter)."""
    prims = np.zeros(2, PRIM_DTYPE)
    mat = MAT_GGX if glossy else MAT_LAMBERT
    _fill_rect(prims[0], (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (rho,) * 3, roughness, mat)
    _fill_rect(prims[1], (0.35, 0.5, 0.35), (0.3, 0.0, 0.0), (0.0, 0.0, 0.3), (0.0,) * 3, 1.0, MAT_BLACK,
               emission=(emission,) * 3)
    origin, top_left, horizontal, vertical = _camera((0.5, 0.9, 0.5), 60.0, width, height)
    # look down (-y): rotate the +z camera frame about x
    top_left = origin + np.array([top_left[0] - origin[0], -1.0, -(top_left[1] - origin[1])])
    vertical = np.array([0.0, 0.0, -vertical[1]])
    return Scene(_header(2, (origin, top_left, horizontal, vertical)), prims, width, height)


def cube_texel_dirs(S: int) -> np.ndarray:
    """Unit direction through the centre of every cube-map texel, (6 S S, 3),
    in the layout the scene blob uses: face 0 +x, 1 -x, 2 +y, 3 -y, 4 +z,
    5 -z; on each face the other two axes in order (a, b), column from a,
    row from b, each spanning [-1, 1]."""
    c = (np.arange(S) + 0.5) / S * 2.0 - 1.0
    b, a = np.meshgrid(c, c, indexing="ij")  # row b, column a
    out = []
    for face in range(6):
        axis, sign = face // 2, (1.0 if face % 2 == 0 else -1.0)
        d = np.zeros((S, S, 3))
        others = [k for k in range(3) if k != axis]
        d[..., axis] = sign
        d[..., others[0]] = a
        d[..., others[1]] = b
        out.append(d.reshape(-1, 3))
    d = np.concatenate(out)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def sky_env(S: int = 64, seed: int = 1) -> np.ndarray:
    """Procedural sky (up = +y): a blue gradient above the horizon, a dim
    ground colour below, and a bright sun lobe in a seeded direction 20-70
    degrees above the horizon.  float32 (6 S S, 4)."""
    rng = np.random.default_rng(seed + 0x5C1)
    d = cube_texel_dirs(S)
    elev = math.radians(float(rng.uniform(20.0, 70.0)))
    azim = float(rng.uniform(0.0, 2.0 * math.pi))
    sun = np.array([math.cos(elev) * math.cos(azim), math.sin(elev), math.cos(elev) * math.sin(azim)])
    up = np.clip(d[:, 1], -1.0, 1.0)
    sky = np.where(up[:, None] > 0.0, np.array([0.35, 0.55, 1.0]) * (0.4 + 0.6 * up[:, None]),
                   np.array([0.12, 0.1, 0.08]))
    lobe = 30.0 * np.clip(d @ sun, 0.0, 1.0) ** 400
    env = np.zeros((d.shape[0], 4), np.float32)
    env[:, :3] = sky + lobe[:, None]
    return env


def uniform_env(S: int, radiance) -> np.ndarray:
    env = np.zeros((6 * S * S, 4), np.float32)
    env[:, :3] = radiance
    return env


def env_scene(width: int, height: int, seed: int = 1, n_prims: int = 64, env_size: int = 64,
              glossy: bool = True) -> Scene:
    """Outdoor scene under an environment map (the Neural Visibility Cache
    workload): a large ground rectangle (y = 0, facing +y) and n_prims - 1
    seeded spheres and rectangles standing on it in [0, 1] x [0, 0.5] x
    [0, 1], under the procedural sky of ``sky_env``; the camera looks down
    at the objects from the front."""
    assert n_prims >= 1
    rng = np.random.default_rng(seed + 0xE1)
    prims = np.zeros(n_prims, PRIM_DTYPE)
    mat = MAT_GGX if glossy else MAT_LAMBERT
    _fill_rect(prims[0], (-20.0, 0.0, -20.0), (0.0, 0.0, 40.0), (40.0, 0.0, 0.0), rng.uniform(0.2, 0.8, 3),
               float(rng.uniform(0.3, 1.0)) if glossy else 1.0, mat)
    for i in range(1, n_prims):
        alb = rng.uniform(0.2, 0.8, 3)
        rough = float(rng.uniform(0.05, 1.0)) if glossy else 1.0
        if i % 2:
            r = float(rng.uniform(0.02, 0.08))
            c = np.array([rng.uniform(0.0, 1.0), r + rng.uniform(0.0, 0.4), rng.uniform(0.0, 1.0)])
            _fill_sphere(prims[i], c, r, alb, rough, mat)
        else:
            nrm = rng.normal(size=3)
            nrm /= np.linalg.norm(nrm)
            t = np.cross(nrm, [1.0, 0.0, 0.0] if abs(nrm[0]) < 0.9 else [0.0, 1.0, 0.0])
            t /= np.linalg.norm(t)
            b = np.cross(nrm, t)
            lu, lv = rng.uniform(0.05, 0.2, 2)
            centre = np.array([rng.uniform(0.0, 1.0), rng.uniform(0.1, 0.5), rng.uniform(0.0, 1.0)])
            corner = centre - 0.5 * t * lu - 0.5 * b * lv
            _fill_rect(prims[i], corner, t * lu, b * lv, alb, rough, mat)
    origin, top_left, horizontal, vertical = _camera((0.5, 0.9, -0.9), 50.0, width, height)
    # tilt the +z camera frame down by 35 degrees about x
    ang = math.radians(35.0)
    rot = np.array([[1.0, 0.0, 0.0], [0.0, math.cos(ang), -math.sin(ang)], [0.0, math.sin(ang), math.cos(ang)]])
    top_left = origin + rot @ (top_left - origin)
    horizontal = rot @ horizontal
    vertical = rot @ vertical
    hd = _header(n_prims, (origin, top_left, horizontal, vertical))
    hd["reserved"][0] = env_size
    sc = Scene(hd, prims, width, height)
    sc.env = sky_env(env_size, seed)
    return sc


def furnace_scene(width: int, height: int, rho: float = 0.5, emission: float = 1.0) -> Scene:
    """White-furnace scene: the camera sits at the centre of a sphere whose
    inner surface is Lambertian with albedo ``rho`` and emits ``emission``
    (both sides).  Every ray from inside hits the sphere."""
    prims = np.zeros(1, PRIM_DTYPE)
    _fill_sphere(prims[0], (0.5, 0.5, 0.5), 0.5, (rho,) * 3, 1.0, MAT_LAMBERT,
                 emission=(emission,) * 3, flags_extra=EMIT_TWO_SIDED)
    cam = _camera((0.5, 0.5, 0.5), 40.0, width, height)
    return Scene(_header(1, cam), prims, width, height)


# ---------------------------------------------------------------------------
# Network configuration and initial parameters
# ---------------------------------------------------------------------------

POS_FREQ, POS_HASHGRID = 0, 1
INPUT_FREQ, INPUT_SH = 0, 1  # network input: frequency encodings, or the paper's SH + phi
OUT_RADIANCE, OUT_VISIBILITY = 0, 1  # cache output: exp radiance, or sigmoid visibility (NVC)


@dataclasses.dataclass
class NetConfig:
    """Hyper-parameters shared by the CUDA path and the oracle."""
    pos_encoding: int = POS_FREQ
    hash_levels: int = 16
    feats_per_level: int = 2
    log2_table: int = 19
    base_res: int = 16
    growth: float = 1.5
    freq_octaves: int = 4
    width: int = 64
    hidden_layers: int = 3
    input_encoding: int = INPUT_FREQ
    output: int = OUT_RADIANCE
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.99
    adam_eps: float = 1e-15
    loss_eps: float = 1e-2
    z_clamp: float = 15.0

    @property
    def n_pos_features(self) -> int:
        if self.pos_encoding == POS_HASHGRID:
            return self.hash_levels * self.feats_per_level
        return 3 * 2 * self.freq_octaves

    @property
    def n_dir_features(self) -> int:
        return 25 if self.input_encoding == INPUT_SH else 2 * 2 * self.freq_octaves

    @property
    def n_surface_features(self) -> int:
        return 3 + 4 + 4 + 4 if self.input_encoding == INPUT_SH else 3 * 2 * self.freq_octaves

    @property
    def n_inputs(self) -> int:
        """Position + direction + per-surface features: frequency encodings of
        (theta, phi) and of the normal, or (INPUT_SH) spherical harmonics of
        the direction and albedo / one-blob normal / one-blob roughness."""
        return self.n_pos_features + self.n_dir_features + self.n_surface_features

    def layer_shapes(self):
        """(fan_out, fan_in) of each weight matrix, input layer first."""
        shapes = [(self.width, self.n_inputs)]
        shapes += [(self.width, self.width)] * (self.hidden_layers - 1)
        shapes.append((3, self.width))
        return shapes

    @property
    def n_mlp_params(self) -> int:
        return sum(o * i + o for o, i in self.layer_shapes())

    @property
    def n_hash_params(self) -> int:
        if self.pos_encoding != POS_HASHGRID:
            return 0
        return self.hash_levels * (1 << self.log2_table) * self.feats_per_level

    @property
    def n_params(self) -> int:
        return self.n_mlp_params + self.n_hash_params


def config_small() -> NetConfig:
    """64x64 correctness workload: frequency encoding of all 8 inputs,
    MLP 64 -> 64 -> 64 -> 64 -> 3, Adam lr 1e-3."""
    return NetConfig(pos_encoding=POS_FREQ, hidden_layers=3, lr=1e-3)


def config_1080p() -> NetConfig:
    """1080p workload: 16-level hash grid (2 features, 2^19 entries, base 16,
    growth 1.5), width 64 with 4 hidden layers, Adam lr 1e-3 (with 1e-2 the
    exp output and Adam's normalised first steps overshoot and the cache
    sinks towards 0 within a few dozen frames on this workload)."""
    return NetConfig(pos_encoding=POS_HASHGRID, hidden_layers=4, lr=1e-3)


def config_paper_1080p() -> NetConfig:
    """The paper's network input on the 1080p workload: 12-level hash grid
    (2 features), spherical harmonics of degree <= 4 of the direction (25)
    and albedo + one-blob normal + one-blob roughness (15), 64 inputs; width
    64 with 4 hidden layers, Adam lr 1e-3."""
    return NetConfig(pos_encoding=POS_HASHGRID, hash_levels=12, hidden_layers=4, input_encoding=INPUT_SH, lr=1e-3)


def init_params(cfg: NetConfig, seed: int = 1) -> np.ndarray:
    """Flat float32 parameter vector: for each layer W (fan_out x fan_in,
    row-major) then b (fan_out), then the hash table [level][entry][feature].
    Weights are Kaiming-uniform, biases zero, hash features U[-1e-4, 1e-4]."""
    rng = np.random.default_rng(seed + 0x5EED)
    parts = []
    for o, i in cfg.layer_shapes():
        bound = math.sqrt(6.0 / i)
        parts.append(rng.uniform(-bound, bound, o * i))
        parts.append(np.zeros(o))
    if cfg.n_hash_params:
        parts.append(rng.uniform(-1e-4, 1e-4, cfg.n_hash_params))
    return np.concatenate(parts).astype(np.float32)


def constant_cache_params(cfg: NetConfig, radiance, seed: int = 1) -> np.ndarray:
    """Parameters whose network outputs exp(ln L) = L for every input: random
    hidden layers, zero output weights, output bias ln(L)."""
    p = init_params(cfg, seed)
    shapes = cfg.layer_shapes()
    off = sum(o * i + o for o, i in shapes[:-1])
    o, i = shapes[-1]
    p[off:off + o * i] = 0.0
    p[off + o * i: off + o * i + o] = np.log(np.asarray(radiance, np.float64) * np.ones(3))
    return p


# ---------------------------------------------------------------------------
# Training-step workload: uniform inputs and an analytic radiance field
# ---------------------------------------------------------------------------

def _unit_sphere(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def analytic_field_params(seed: int = 7):
    """Eight lobes: amplitude a_k (RGB, U[0.1, 2]), sharpness kappa_k
    (U[2, 50]), axis mu_k (uniform on the sphere), spatial frequency f_k
    (U[1, 4]^3) and phase psi_k (U[0, 2 pi])."""
    rng = np.random.default_rng(seed)
    return dict(
        a=rng.uniform(0.1, 2.0, (8, 3)),
        kappa=rng.uniform(2.0, 50.0, 8),
        mu=_unit_sphere(rng, 8),
        f=rng.uniform(1.0, 4.0, (8, 3)),
        psi=rng.uniform(0.0, 2.0 * math.pi, 8),
    )


def analytic_field(x: np.ndarray, w: np.ndarray, fp) -> np.ndarray:
    """L(x, w) = sum_k a_k exp(kappa_k (w . mu_k - 1)) (1 + 0.5 sin(2 pi f_k . x + psi_k))."""
    cosang = w @ fp["mu"].T                                     # (n, 8)
    lobe = np.exp(fp["kappa"][None, :] * (cosang - 1.0))
    mod = 1.0 + 0.5 * np.sin(2.0 * math.pi * (x @ fp["f"].T) + fp["psi"][None, :])
    return (lobe * mod) @ fp["a"]                                # (n, 3)


def training_batch(n: int, seed: int = 3, field_seed: int = 7):
    """Seeded training batch: records with x ~ U[0,1]^3, normal uniform on
    the sphere, albedo ~ U[0.2,0.8]^3 and roughness ~ U[0.05,1] (the scene
    family's materials), directions uniform on the sphere, targets from the
    analytic field (of x and the direction only).  Returns
    (records[RECORD_DTYPE], dirs f32 (n,3), targets f32 (n,3))."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, (n, 3))
    nrm = _unit_sphere(rng, n)
    w = _unit_sphere(rng, n)
    rec = np.zeros(n, RECORD_DTYPE)
    rec["p"] = x
    rec["n"] = nrm
    rec["wo"] = nrm
    rec["albedo"] = rng.uniform(0.2, 0.8, (n, 3))
    rec["roughness"] = rng.uniform(0.05, 1.0, n)
    rec["prim"] = 0
    rec["flags"] = 1 | (MAT_LAMBERT << 1)
    tgt = analytic_field(x, w, analytic_field_params(field_seed))
    return rec, w.astype(np.float32), tgt.astype(np.float32)


def random_query_rows(n: int, seed: int = 5):
    """Arbitrary cache queries: records with x ~ U[0,1]^3, normals and
    directions uniform on the sphere."""
    rec, dirs, _ = training_batch(n, seed)
    return rec, dirs
