"""CPU ORACLE -- test infrastructure only.

A plain, slow, obviously-correct CPU statement of what the rendering method computes, used
to judge the CUDA library.  Only the tests, the smoke check and the benchmark's CPU-baseline
leg may import it; the library never does and shares no code with it.

Parts:
  * oracle.c (C, built here with -ffp-contract=off): the rasterizer's render and resolve
    passes (Sec. 3.2), packing of the G-buffer into the network input, and a Gaussian splat
    renderer standing in for the paper's Gaussian Renderer (Sec. 4.2).
  * unet.py: the fixed U-Net forward/backward, L1 loss and Adam in float64 (Sec. 3.3).
  * metrics.py: PSNR and SSIM (Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import metrics, unet  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
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
        P, I, I64, U64, F, D = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                ctypes.c_float, ctypes.c_double)
        lib.oracle_visibility.argtypes = [P, U64, P, I, I, F, F, P]
        lib.oracle_visibility_mt.argtypes = [P, U64, P, I, I, F, F, P]
        lib.oracle_resolve.argtypes = [P, I64, P, I64, I, P, P, P]
        lib.oracle_pack.argtypes = [P, P, P, I, I, I, I, I, P, P, P, P, P, F, F, I, I, F, P]
        lib.oracle_splat.argtypes = [P, U64, P, I, I, F, F, P, D, D, P]
        lib.oracle_splat_aniso.argtypes = [P, U64, P, I, I, F, F, P, P, D, D, D, P]
        lib.oracle_bf16_array.argtypes = [P, I64, P]
        lib.oracle_e4m3_array.argtypes = [P, I64, P]
        _lib = lib
    return _lib


def _p(a):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def visibility(xyz: np.ndarray, view, threads: str = "one") -> np.ndarray:
    """Per-pixel minimum key (bits(depth) << 32 | index) over all points; ~0 where empty.
    threads="all": the same keys from per-thread minima combined by a minimum."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    m = np.ascontiguousarray(view.viewproj, np.float32)
    key = np.empty((view.height, view.width), np.uint64)
    fn = _L().oracle_visibility_mt if threads == "all" else _L().oracle_visibility
    fn(_p(xyz), xyz.shape[0], _p(m), view.width, view.height, float(view.znear),
       float(view.zfar), _p(key))
    return key


def resolve(key: np.ndarray, attr: np.ndarray, k: int):
    """(depth u32 [H,W], mask u8 [H,W], attribute words u32 [K,H,W]) from the key image."""
    key = np.ascontiguousarray(key, np.uint64)
    attr = np.ascontiguousarray(attr, np.uint32)
    h, w = key.shape
    depth = np.empty((h, w), np.uint32)
    mask = np.empty((h, w), np.uint8)
    gattr = np.empty((k, h, w), np.uint32)
    _L().oracle_resolve(_p(key), h * w, _p(attr), attr.shape[1], k, _p(depth), _p(mask), _p(gattr))
    return depth, mask, gattr


def rasterize(scene, view):
    key = visibility(scene.xyz, view)
    return (key,) + resolve(key, scene.attr, scene.n_words)


def pack(depth, mask, gattr, channels, d_scale: float, d_offset: float, hn: int, wn: int,
         cpad: int, out_fmt: int = 0, in_scale_inv: float = 1.0) -> np.ndarray:
    """Network input [Hn, Wn, cpad] (float32, bf16 bits as uint16, or e4m3 bits as uint8)."""
    h, w = depth.shape
    nch = len(channels)
    assert nch + 2 <= cpad
    cw = np.array([c.word for c in channels], np.int32)
    cf = np.array([c.fmt for c in channels], np.int32)
    cc = np.array([c.comp for c in channels], np.int32)
    cs = np.array([c.scale for c in channels], np.float32)
    co = np.array([c.offset for c in channels], np.float32)
    dt = {0: np.float32, 1: np.uint16, 2: np.uint8}[out_fmt]
    out = np.empty((hn, wn, cpad), dt)
    _L().oracle_pack(_p(np.ascontiguousarray(depth, np.uint32)), _p(np.ascontiguousarray(mask, np.uint8)),
                     _p(np.ascontiguousarray(gattr, np.uint32)), h, w, hn, wn, nch, _p(cw), _p(cf),
                     _p(cc), _p(cs), _p(co), float(d_scale), float(d_offset), cpad, out_fmt,
                     float(in_scale_inv), _p(out))
    return out


def splat_aniso(xyz: np.ndarray, view, colour: np.ndarray, velocity: np.ndarray, r0: float,
                stretch: float, alpha: float = 0.6):
    """Elongated Gaussians (covariance r0^2 R diag(s^2, 1, 1) R^T along each point's velocity,
    projected with the screen map's Jacobian), composited front to back -> float64 RGB [H, W, 3].
    Serial: for pins and small stylised targets."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    colour = np.ascontiguousarray(colour, np.float32)
    velocity = np.ascontiguousarray(velocity, np.float32)
    m = np.ascontiguousarray(view.viewproj, np.float32)
    out = np.empty((view.height, view.width, 3), np.float64)
    _L().oracle_splat_aniso(_p(xyz), xyz.shape[0], _p(m), view.width, view.height, float(view.znear),
                            float(view.zfar), _p(colour), _p(velocity), float(r0), float(stretch),
                            float(alpha), _p(out))
    return out


def bf16_bits(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    _L().oracle_bf16_array(_p(x), x.size, _p(out))
    return out


def bf16_value(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, np.uint32) << 16).view(np.float32)


def e4m3_bits(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty(x.shape, np.uint8)
    _L().oracle_e4m3_array(_p(x), x.size, _p(out))
    return out


def e4m3_value(bits: np.ndarray) -> np.ndarray:
    """Decode E4M3 bits to float64 from the format's definition."""
    b = np.asarray(bits, np.uint8).astype(np.int64)
    s = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    m = b & 0x7
    val = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * np.exp2(e - 7.0))
    val = np.where((e == 15) & (m == 7), np.nan, val)
    return s * val


def splat(xyz: np.ndarray, view, colour: np.ndarray, sigma: float = 1.5, alpha: float = 0.6):
    """Front-to-back alpha-composited isotropic Gaussians -> float64 RGB [H, W, 3]."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    colour = np.ascontiguousarray(colour, np.float32)
    m = np.ascontiguousarray(view.viewproj, np.float32)
    out = np.empty((view.height, view.width, 3), np.float64)
    _L().oracle_splat(_p(xyz), xyz.shape[0], _p(m), view.width, view.height, float(view.znear),
                      float(view.zfar), _p(colour), float(sigma), float(alpha), _p(out))
    return out


# Derived channel formats of the library's pack descriptor (Sec. 4.5 "Vel2D", Sec. 3.2 splat
# radius); the values follow include/nrv.h's numbering of nrv_fmt.
VEL2D_X, VEL2D_Y, VEL2D_ANGLE, VEL2D_MAG, SPLAT_RADIUS = 3, 4, 5, 6, 7


def derived_channel(key: np.ndarray, xyz: np.ndarray, attr: np.ndarray, view, fmt: int,
                    word: int) -> np.ndarray:
    """FP64 value of one derived channel at every pixel of a key image (NaN where empty).

    Vel2D (Sec. 4.5): the velocity v (record words word..word+2, FP32) of the winning point p,
    perspective-projected: v' = J v with J the Jacobian of the screen map
    s(p) = ((c_x / c_w + 1) W/2, (1 - c_y / c_w) H/2), c = M (p, 1), so
        J_x = (W/2) (M_0 c_w - c_x M_3) / c_w^2,   J_y = -(H/2) (M_1 c_w - c_y M_3) / c_w^2
    (M_r the first three entries of row r); the channels are v'_x, v'_y, the angle atan2(v'_y,
    v'_x) of v' in the image plane and |v'|.  Splat radius (Sec. 3.2, terrain): the world
    radius r (record word `word`, FP32) in pixels, r (H/2) |M_1| / c_w."""
    key = np.asarray(key, np.uint64)
    hit = key != np.uint64(0xFFFFFFFFFFFFFFFF)
    idx = (key[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    M = np.asarray(view.viewproj, np.float32).astype(np.float64).reshape(4, 4)
    p = np.asarray(xyz, np.float32)[idx].astype(np.float64)
    rec = np.asarray(attr, np.uint32)[idx]
    ph = np.concatenate([p, np.ones((len(p), 1))], 1)
    c = ph @ M.T
    cx, cy, cw = c[:, 0], c[:, 1], c[:, 3]
    out = np.full(key.shape, np.nan)
    if fmt == SPLAT_RADIUS:
        r = rec[:, word].view(np.float32).astype(np.float64)
        out[hit] = r * (view.height / 2.0) * np.linalg.norm(M[1, :3]) / cw
        return out
    v = np.ascontiguousarray(rec[:, word:word + 3]).view(np.float32).astype(np.float64)
    jx = (view.width / 2.0) * (M[0, :3][None] * cw[:, None] - cx[:, None] * M[3, :3][None]) / cw[:, None] ** 2
    jy = -(view.height / 2.0) * (M[1, :3][None] * cw[:, None] - cy[:, None] * M[3, :3][None]) / cw[:, None] ** 2
    vx, vy = (jx * v).sum(1), (jy * v).sum(1)
    out[hit] = {VEL2D_X: vx, VEL2D_Y: vy, VEL2D_ANGLE: np.arctan2(vy, vx),
                VEL2D_MAG: np.hypot(vx, vy)}[fmt]
    return out
