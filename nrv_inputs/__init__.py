"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the CPU oracle.

This module generates inputs only: point clouds with their attribute records,
camera matrices, per-channel normalisation constants and Xavier-uniform weight
tensors.  It holds none of the rendering method's arithmetic; the projection,
visibility, resolve, packing and network math live separately in the CUDA
library and in the oracle, which share no code.

Scenes follow the four synthetic workloads that stand in for the paper's
datasets (Sec. 4.1): a uniform cube, a static Rankine-vortex field (vector-field
data like Hurricane), RK4 particle trajectories through a sum of vortices
(trajectory data like Storms), and an fBm terrain scan (like Morro Bay).
Cameras follow the paper's training setup: 60 degree field of view with the
near and far planes at 0.1 and 2e5 (Sec. 3.3), and the hemisphere viewpoint
strategy (Appendix A).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libnrvinputs.so")
_lib = None

FMT_F32, FMT_U32, FMT_U8X4 = 0, 1, 2
ZNEAR, ZFAR, FOVY_DEG = 0.1, 2.0e5, 60.0


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library beside it (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I64, U64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.nrvi_bits.restype = U64
        lib.nrvi_bits.argtypes = [U64, U64, U64]
        lib.nrvi_uniform.restype = D
        lib.nrvi_uniform.argtypes = [U64, U64, U64]
        lib.nrvi_normal.restype = D
        lib.nrvi_normal.argtypes = [U64, U64, U64]
        lib.nrvi_fill_uniform.argtypes = [U64, U64, I64, D, D, P, I64]
        lib.nrvi_fill_normal.argtypes = [U64, U64, I64, P, I64]
        lib.nrvi_cube_points.argtypes = [U64, I64, P]
        lib.nrvi_vortex_grid.argtypes = [I64, U64, D, P, P, I64]
        lib.nrvi_vortex_params.argtypes = [U64, ctypes.c_int, P]
        lib.nrvi_trajectories.argtypes = [I64, I64, D, U64, P, ctypes.c_int, P, P, I64]
        lib.nrvi_terrain.argtypes = [I64, D, U64, P, P, I64]
        lib.nrvi_terrain_height.restype = D
        lib.nrvi_terrain_height.argtypes = [U64, D, D]
        lib.nrvi_channel_moments.argtypes = [P, I64, I64, I64, ctypes.c_int, ctypes.c_int, P, P]
        lib.nrvi_bbox.argtypes = [P, I64, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def uniform(seed: int, stream: int, index: int) -> float:
    return _L().nrvi_uniform(seed, stream, index)


def uniform_array(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(n, np.float32)
    _L().nrvi_fill_uniform(seed, stream, n, lo, hi, _p(out), 1)
    return out


def normal_array(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _L().nrvi_fill_normal(seed, stream, n, _p(out), 1)
    return out


# --------------------------------------------------------------------------- scenes

@dataclass
class Channel:
    """One scalar network channel read from a record word (fmt: f32, u32 or byte of u8x4)."""
    word: int
    fmt: int
    comp: int = 0
    scale: float = 1.0
    offset: float = 0.0


@dataclass
class Scene:
    name: str
    xyz: np.ndarray            # float32 [N, 3], C-contiguous
    attr: np.ndarray           # uint32 [N, stride_words]
    n_words: int               # meaningful words per record (K in the G-buffer)
    channels: list = field(default_factory=list)   # list[Channel], normalisation filled in
    colour_channel: int = 0    # index into channels used by the colour map

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def stride_words(self) -> int:
        return int(self.attr.shape[1])

    def bbox(self):
        lo = np.empty(3, np.float64)
        hi = np.empty(3, np.float64)
        _L().nrvi_bbox(_p(self.xyz), self.n, _p(lo), _p(hi))
        return lo, hi

    def subset(self, idx: np.ndarray, name: str | None = None) -> "Scene":
        return Scene(name or self.name + "-subset", np.ascontiguousarray(self.xyz[idx]),
                     np.ascontiguousarray(self.attr[idx]), self.n_words,
                     [Channel(**vars(c)) for c in self.channels], self.colour_channel)


def _normalise(scene: Scene) -> Scene:
    """scale = 1/std, offset = -mean/std per channel, from double moments over all points."""
    for ch in scene.channels:
        m = np.zeros(1, np.float64)
        s = np.zeros(1, np.float64)
        _L().nrvi_channel_moments(_p(scene.attr), scene.n, scene.stride_words, ch.word, ch.fmt,
                                  ch.comp, _p(m), _p(s))
        sd = float(s[0]) if s[0] > 0 else 1.0
        ch.scale = float(np.float32(1.0 / sd))
        ch.offset = float(np.float32(-float(m[0]) / sd))
    return scene


def cube_scene(n: int = 1_000_000, k: int = 3, seed: int = 0) -> Scene:
    """n points uniform in [0,1)^3 with k f32 attributes ~ N(0,1); records of 4 or 8 words."""
    xyz = np.empty((n, 3), np.float32)
    _L().nrvi_cube_points(seed, n, _p(xyz))
    sw = 4 if k <= 4 else 8
    attr = np.zeros((n, sw), np.uint32)
    for j in range(k):
        col = normal_array(seed, 10 + j, n)
        attr[:, j] = col.view(np.uint32)
    sc = Scene(f"cube-{n}", xyz, attr, k, [Channel(j, FMT_F32) for j in range(k)], 0)
    return _normalise(sc)


def vortex_grid_scene(g: int = 368, seed: int = 1, sigma: float = 0.05) -> Scene:
    """Jittered g^3 grid with a Rankine vortex velocity (+noise), speed and pressure (K=5)."""
    n = g ** 3
    xyz = np.empty((n, 3), np.float32)
    attr = np.empty((n, 8), np.uint32)
    _L().nrvi_vortex_grid(g, seed, sigma, _p(xyz), _p(attr), 8)
    sc = Scene(f"vortex-grid-{g}", xyz, attr, 5, [Channel(j, FMT_F32) for j in range(5)], 3)
    return _normalise(sc)


def vortex_params(seed: int, nv: int = 8) -> np.ndarray:
    out = np.empty((nv, 8), np.float64)
    _L().nrvi_vortex_params(seed, nv, _p(out))
    return out


def trajectory_scene(n_particles: int = 1_000_000, n_steps: int = 350, dt: float = 0.01,
                     seed: int = 2, n_vortices: int = 8) -> Scene:
    """Particle-major RK4 trajectories; records (t f32, speed f32, id u32, pad), K=3."""
    n = n_particles * n_steps
    vort = vortex_params(seed, n_vortices)
    xyz = np.empty((n, 3), np.float32)
    attr = np.empty((n, 4), np.uint32)
    _L().nrvi_trajectories(n_particles, n_steps, dt, seed, _p(vort), n_vortices, _p(xyz),
                           _p(attr), 4)
    chans = [Channel(0, FMT_F32), Channel(1, FMT_F32), Channel(2, FMT_U32)]
    sc = Scene(f"trajectories-{n_particles}x{n_steps}", xyz, attr, 3, chans, 1)
    return _normalise(sc)


def terrain_scene(g: int = 14142, extent: float = 1.0e4, seed: int = 7) -> Scene:
    """fBm terrain in Morton order of 64x64 cells; records (RGBA8, intensity f32), K=2 words,
    4 network channels (R, G, B bytes and intensity)."""
    n = g * g
    xyz = np.empty((n, 3), np.float32)
    attr = np.empty((n, 2), np.uint32)
    _L().nrvi_terrain(g, extent, seed, _p(xyz), _p(attr), 2)
    chans = [Channel(0, FMT_U8X4, 0), Channel(0, FMT_U8X4, 1), Channel(0, FMT_U8X4, 2),
             Channel(1, FMT_F32)]
    sc = Scene(f"terrain-{g}", xyz, attr, 2, chans, 0)
    return _normalise(sc)


def terrain_height(x: float, z: float, seed: int = 7) -> float:
    return _L().nrvi_terrain_height(seed, x, z)


def shuffled(scene: Scene, seed: int = 99) -> Scene:
    """The same scene in a seeded random point order (the adversarial order for binning)."""
    perm = np.random.default_rng(seed).permutation(scene.n)
    return scene.subset(perm, scene.name + "-shuffled")


# --------------------------------------------------------------------------- cameras

@dataclass
class View:
    viewproj: np.ndarray   # float32 [16], row-major; clip = M @ [x y z 1]
    width: int
    height: int
    znear: float = ZNEAR
    zfar: float = ZFAR
    eye: tuple = (0.0, 0.0, 0.0)
    view: np.ndarray | None = None   # float64 [4,4] world->eye, kept for depth ranges


def look_at(eye, target, up) -> np.ndarray:
    """OpenGL-style world->eye matrix (camera looks down -z in eye space)."""
    e, t, u = (np.asarray(v, np.float64) for v in (eye, target, up))
    f = t - e
    f /= np.linalg.norm(f)
    s = np.cross(f, u)
    s /= np.linalg.norm(s)
    uu = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, uu, -f
    m[:3, 3] = -m[:3, :3] @ e
    return m


def perspective(fovy_deg: float, aspect: float, znear: float, zfar: float) -> np.ndarray:
    """OpenGL-style projection; the clip w row is (0, 0, -1, 0) so w = eye-space depth."""
    f = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    p = np.zeros((4, 4))
    p[0, 0] = f / aspect
    p[1, 1] = f
    p[2, 2] = (zfar + znear) / (znear - zfar)
    p[2, 3] = 2.0 * zfar * znear / (znear - zfar)
    p[3, 2] = -1.0
    return p


def make_view(eye, target, width: int, height: int, up=(0.0, 1.0, 0.0), fovy_deg: float = FOVY_DEG,
              znear: float = ZNEAR, zfar: float = ZFAR) -> View:
    """The view-projection is built in double and rounded to float32 once."""
    v = look_at(eye, target, up)
    m = perspective(fovy_deg, width / height, znear, zfar) @ v
    return View(np.ascontiguousarray(m.astype(np.float32).reshape(16)), width, height, znear, zfar,
                tuple(float(x) for x in eye), v)


def cube_view(width: int = 512, height: int = 512) -> View:
    """Camera at (0.5, 0.5, 3) looking at the cube centre, +y up."""
    return make_view((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), width, height)


def fitted_view(scene: Scene, width: int = 1920, height: int = 1080, direction=(0.0, 0.0, 1.0)) -> View:
    """Camera on `direction` from the bbox centre, far enough that the bbox sphere fits the
    vertical field of view."""
    lo, hi = scene.bbox()
    c = 0.5 * (lo + hi)
    r = 0.5 * float(np.linalg.norm(hi - lo))
    d = np.asarray(direction, np.float64)
    d /= np.linalg.norm(d)
    dist = r / math.sin(math.radians(FOVY_DEG) / 2.0)
    return make_view(tuple(c + d * dist), tuple(c), width, height)


def hemisphere_views(scene: Scene, n: int, width: int, height: int, seed: int = 5) -> list:
    """Seeded cameras on the hemisphere of radius 0.75 x bbox diagonal about the bbox centre
    (Appendix A), looking at the centre; theta/phi on the pi/8, pi/16 lattice of that strategy,
    picked in a seeded order."""
    lo, hi = scene.bbox()
    c = 0.5 * (lo + hi)
    r = 0.75 * float(np.linalg.norm(hi - lo))
    lattice = [(ti * math.pi / 8.0, pj * math.pi / 16.0) for ti in range(16) for pj in range(1, 8)]
    order = np.argsort([uniform(seed, 300, i) for i in range(len(lattice))], kind="stable")
    views = []
    for k in range(n):
        th, ph = lattice[int(order[k % len(lattice)])]
        # polar angle phi from the +y (up) axis, azimuth theta in the x-z plane
        eye = c + r * np.array([math.sin(ph) * math.cos(th), math.cos(ph), math.sin(ph) * math.sin(th)])
        views.append(make_view(tuple(eye), tuple(c), width, height))
    return views


def orbit_views(scene: Scene, sizes, seed: int = 11, stereo_pairs: int = 0, ipd: float = 0.065):
    """Seeded orbit cameras around the terrain centre for a batch of views of the given sizes;
    the first 2*stereo_pairs views are left/right eyes sharing one orbit position."""
    lo, hi = scene.bbox()
    c = 0.5 * (lo + hi)
    ext = float(max(hi[0] - lo[0], hi[2] - lo[2]))
    views = []
    k = 0
    while len(views) < len(sizes):
        th = 2.0 * math.pi * uniform(seed, 400, k)
        rad = ext * (0.55 + 0.25 * uniform(seed, 401, k))
        hgt = ext * (0.25 + 0.2 * uniform(seed, 402, k))
        eye = np.array([c[0] + rad * math.cos(th), c[1] + hgt, c[2] + rad * math.sin(th)])
        tgt = c.copy()
        if len(views) < 2 * stereo_pairs:
            fwd = tgt - eye
            side = np.cross(fwd, [0.0, 1.0, 0.0])
            side /= np.linalg.norm(side)
            for s in (-0.5, 0.5):
                w, h = sizes[len(views)]
                views.append(make_view(tuple(eye + s * ipd * side), tuple(tgt + s * ipd * side), w, h))
        else:
            w, h = sizes[len(views)]
            views.append(make_view(tuple(eye), tuple(tgt), w, h))
        k += 1
    return views


def depth_normalisation(scene: Scene, view: View):
    """(scale, offset) for the depth channel: 1/(far-near) and -near/(far-near) over the eye-space
    depths of the scene bbox corners, clamped to the view's near plane; float32 values."""
    lo, hi = scene.bbox()
    corners = np.array([[x, y, z, 1.0] for x in (lo[0], hi[0]) for y in (lo[1], hi[1])
                        for z in (lo[2], hi[2])])
    d = -(corners @ view.view[2])
    dn = max(float(d.min()), view.znear)
    df = max(float(d.max()), dn + 1e-6)
    s = 1.0 / (df - dn)
    return float(np.float32(s)), float(np.float32(-dn * s))


# --------------------------------------------------------------------------- weights

def xavier_uniform(seed: int, stream: int, shape, fan_in: int, fan_out: int) -> np.ndarray:
    """Xavier/Glorot uniform: U(-b, b), b = sqrt(6/(fan_in+fan_out)), element i from
    uniform(seed, stream, i) in C order; returned as float32."""
    n = int(np.prod(shape))
    b = math.sqrt(6.0 / (fan_in + fan_out))
    u = np.empty(n, np.float32)
    _L().nrvi_fill_uniform(seed, stream, n, -b, b, _p(u), 1)
    return u.reshape(shape)


def random_crops(seed: int, step: int, batch: int, n_views: int, height: int, width: int, crop: int):
    """Seeded (view, y0, x0) triples for one training step."""
    out = []
    for b in range(batch):
        i = step * batch + b
        v = int(uniform(seed, 500, i) * n_views)
        y = int(uniform(seed, 501, i) * (height - crop + 1))
        x = int(uniform(seed, 502, i) * (width - crop + 1))
        out.append((v, y, x))
    return out


# --------------------------------------------------------------------------- transfer function

# Five-stop piecewise-linear colour map (user-defined transfer function, Sec. 3.2); the stops
# are samples of a perceptually ordered blue-green-yellow ramp.
COLOUR_STOPS = np.array([[0.267, 0.005, 0.329], [0.229, 0.322, 0.546], [0.128, 0.567, 0.551],
                         [0.369, 0.789, 0.383], [0.993, 0.906, 0.144]], np.float64)


def colour_map(t: np.ndarray) -> np.ndarray:
    """t in [0, 1] (clamped) -> RGB float32 by linear interpolation between the five stops."""
    t = np.clip(np.asarray(t, np.float64), 0.0, 1.0) * 4.0
    i = np.minimum(t.astype(np.int64), 3)
    f = (t - i)[..., None]
    return (COLOUR_STOPS[i] * (1.0 - f) + COLOUR_STOPS[i + 1] * f).astype(np.float32)


def point_colours(scene: Scene) -> np.ndarray:
    """Per-point RGB in [0,1] from the scene's transfer function: stored RGB bytes for
    u8x4 colour channels, otherwise the colour map of the z-scored colour channel mapped
    from [-2, 2] to [0, 1]."""
    ch = scene.channels[scene.colour_channel]
    w = scene.attr[:, ch.word]
    if ch.fmt == FMT_U8X4:
        rgb = np.stack([(w >> (8 * c)) & 255 for c in range(3)], axis=-1)
        return (rgb.astype(np.float32) / np.float32(255.0))
    v = w.view(np.float32).astype(np.float64) if ch.fmt == FMT_F32 else w.astype(np.float64)
    z = v * ch.scale + ch.offset
    return colour_map((z + 2.0) / 4.0)
