"""Python binding of libnrv (include/nrv.h): ctypes declarations with the C names, plus thin
helpers that marshal torch CUDA tensors into the C structs.  Every step of the rendering path
runs in the library's CUDA kernels; nothing here computes.  There is no fallback: if the
library is missing or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnrv.so")

NRV_OK, NRV_ERR_ARG, NRV_ERR_CUDA, NRV_ERR_OOM, NRV_ERR_TIMEOUT, NRV_ERR_UNSUPPORTED, NRV_ERR_STATE = range(7)
NRV_F32, NRV_U32, NRV_U8X4 = 0, 1, 2
NRV_VEL2D_X, NRV_VEL2D_Y, NRV_VEL2D_ANGLE, NRV_VEL2D_MAG, NRV_SPLAT_RADIUS = 3, 4, 5, 6, 7
PREC_F32, PREC_BF16, PREC_FP8_E4M3, PREC_FP8 = 0, 1, 2, 3
STATUS_NAMES = ["NRV_OK", "NRV_ERR_ARG", "NRV_ERR_CUDA", "NRV_ERR_OOM", "NRV_ERR_TIMEOUT",
                "NRV_ERR_UNSUPPORTED", "NRV_ERR_STATE"]


class NrvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class nrv_scene_desc(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_uint64), ("d_xyz", ctypes.c_void_p), ("d_attr", ctypes.c_void_p),
                ("stride_words", ctypes.c_int), ("n_words", ctypes.c_int),
                ("point_stride", ctypes.c_int), ("index_base", ctypes.c_uint64)]


class nrv_view(ctypes.Structure):
    _fields_ = [("viewproj", ctypes.c_float * 16), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("znear", ctypes.c_float), ("zfar", ctypes.c_float)]


class nrv_gbuffer(ctypes.Structure):
    _fields_ = [("d_key", ctypes.c_void_p), ("d_depth", ctypes.c_void_p), ("d_mask", ctypes.c_void_p),
                ("d_attr", ctypes.c_void_p)]


class nrv_pack_desc(ctypes.Structure):
    _fields_ = [("n_channels", ctypes.c_int), ("word", ctypes.c_int * 6), ("fmt", ctypes.c_int * 6),
                ("comp", ctypes.c_int * 6), ("scale", ctypes.c_float * 6), ("offset", ctypes.c_float * 6),
                ("depth_scale", ctypes.c_float), ("depth_offset", ctypes.c_float)]


class nrv_loss_weights(ctypes.Structure):
    _fields_ = [("l1", ctypes.c_float), ("l2", ctypes.c_float), ("tv", ctypes.c_float)]


class nrv_layer_info(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 8), ("kind", ctypes.c_int), ("c_in", ctypes.c_int),
                ("c_out", ctypes.c_int), ("weight_offset", ctypes.c_int64), ("bias_offset", ctypes.c_int64)]


P, I, I64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
# name -> (restype, argtypes): the exported surface of include/nrv.h
SIGNATURES = {
    "nrv_last_error": (ctypes.c_char_p, []),
    "nrv_version": (I, []),
    "nrv_launch_count": (ctypes.c_uint64, []),
    "nrv_render_variants": (I, [I]),
    "nrv_pad8": (I, [I]),
    "nrv_netin_channels": (I, [I]),
    "nrv_create_scene": (I, [ctypes.POINTER(nrv_scene_desc), ctypes.POINTER(P)]),
    "nrv_destroy_scene": (I, [P]),
    "nrv_scene_refresh": (I, [P]),
    "nrv_rasterize": (I, [P, ctypes.POINTER(nrv_view), I, ctypes.POINTER(nrv_gbuffer), P]),
    "nrv_pack": (I, [ctypes.POINTER(nrv_gbuffer), I, I, ctypes.POINTER(nrv_pack_desc), I, F, P, P]),
    "nrv_resolve": (I, [P, ctypes.POINTER(nrv_view), P, ctypes.POINTER(nrv_gbuffer), P]),
    "nrv_keys_flip_sign": (I, [P, I64, P]),
    "nrv_resolve_pack": (I, [P, ctypes.POINTER(nrv_view), P, ctypes.POINTER(nrv_pack_desc), I, F, P, P]),
    "nrv_net_num_layers": (I, []),
    "nrv_net_layer": (I, [I, I, ctypes.POINTER(nrv_layer_info)]),
    "nrv_net_param_count": (I, [I, ctypes.POINTER(I64)]),
    "nrv_create_net": (I, [I, ctypes.POINTER(P)]),
    "nrv_destroy_net": (I, [P]),
    "nrv_net_set_params": (I, [P, P, P]),
    "nrv_net_init_params": (I, [P, ctypes.c_uint64, P, P]),
    "nrv_net_get_params": (I, [P, P, P]),
    "nrv_net_save": (I, [P, ctypes.c_char_p, P]),
    "nrv_net_load": (I, [P, ctypes.c_char_p, P]),
    "nrv_net_set_act_scales": (I, [P, ctypes.POINTER(F), I, P]),
    "nrv_net_get_act_scales": (I, [P, ctypes.POINTER(F), I]),
    "nrv_net_calibrate": (I, [P, P, I, I, I, P]),
    "nrv_shade": (I, [P, P, I, I, I, I, P, P]),
    "nrv_net_layer_backend": (I, [P, I]),
    "nrv_net_run_layer": (I, [P, I, P, P, I, I, I, I, P, P]),
    "nrv_net_layer_wgrad": (I, [P, I, P, P, P, I, I, I, I, P, P]),
    "nrv_net_layer_dgrad": (I, [P, I, P, P, I, I, I, I, P, P]),
    "nrv_probe_ffma": (I, [P, I, I, P]),
    "nrv_probe_atomic_min": (I, [P, I64, I64, ctypes.c_uint64, P]),
    "nrv_net_forward_train": (I, [P, P, I, I, I, I, P, P]),
    "nrv_net_backward": (I, [P, P, P, P]),
    "nrv_l1_loss": (I, [P, P, I64, P, P, P]),
    "nrv_l1_loss_noalloc": (I, [P, P, I64, P, P, P]),
    "nrv_adam_step": (I, [P, P, P, P, I64, I, F, F, F, F, P]),
    "nrv_recon_loss": (I, [P, P, I, I, I, ctypes.POINTER(nrv_loss_weights), P, P, P]),
    "nrv_net_set_loss": (I, [P, ctypes.POINTER(nrv_loss_weights)]),
    "nrv_train_step": (I, [P, P, P, P, P, I, F, P, P, I, I, I, I, P, P]),
    "nrv_render_batch": (I, [P, P, ctypes.POINTER(nrv_pack_desc), ctypes.POINTER(nrv_view), I,
                             ctypes.POINTER(P), I, F, P]),
    "nrv_set_profiling": (I, [I]),
    "nrv_get_timings": (I, [ctypes.POINTER(F), I]),
    "nrv_sync_status": (I, [P]),
    "nrv_gnet_num_layers": (I, []),
    "nrv_gnet_layer": (I, [I, I, ctypes.POINTER(nrv_layer_info)]),
    "nrv_gnet_param_count": (I, [I, ctypes.POINTER(I64)]),
    "nrv_gnet_create": (I, [I, ctypes.POINTER(P)]),
    "nrv_gnet_destroy": (I, [P]),
    "nrv_gnet_set_params": (I, [P, P, P]),
    "nrv_gnet_shade": (I, [P, P, I, I, I, P, P]),
    "nrv_gnet_run_layer": (I, [P, I, P, P, I, I, I, P, P]),
    "nrv_tune_load": (I, [ctypes.c_char_p]),
    "nrv_tune_save": (I, [ctypes.c_char_p]),
    "nrv_tune_count": (I, []),
    "nrv_tune_timings": (ctypes.c_uint64, []),
}

_lib = None


def lib():
    """Load libnrv.so (built in-tree by build_lib.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libnrv.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != NRV_OK:
        raise NrvError(status, lib().nrv_last_error().decode(errors="replace"))


def _ptr(t) -> int | None:
    if t is None:
        return None
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "need a contiguous CUDA tensor"
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_view(v) -> nrv_view:
    """From any object with viewproj (16 floats), width, height, znear, zfar."""
    cv = nrv_view()
    m = np.asarray(v.viewproj, np.float32).reshape(16)
    for i in range(16):
        cv.viewproj[i] = float(m[i])
    cv.width, cv.height, cv.znear, cv.zfar = int(v.width), int(v.height), float(v.znear), float(v.zfar)
    return cv


def make_pack_desc(channels, depth_scale: float, depth_offset: float) -> nrv_pack_desc:
    d = nrv_pack_desc()
    d.n_channels = len(channels)
    for j, c in enumerate(channels):
        d.word[j], d.fmt[j], d.comp[j] = int(c.word), int(c.fmt), int(c.comp)
        d.scale[j], d.offset[j] = float(c.scale), float(c.offset)
    d.depth_scale, d.depth_offset = float(depth_scale), float(depth_offset)
    return d


class Scene:
    """A scene handle borrowing device tensors xyz [N,3] float32 and attr [N,S] int32/uint32."""

    def __init__(self, xyz, attr, n_words: int, index_base: int = 0, point_stride: int = 1):
        """point_stride S > 1: the scene is every S-th point of xyz/attr (a masked render pass
        over a subset, e.g. glyph points); keys then carry the index in the full arrays."""
        self.xyz, self.attr = xyz, attr      # keep the borrowed memory alive
        n = int(xyz.shape[0])
        if point_stride > 1:
            n = (n + point_stride - 1) // point_stride
        d = nrv_scene_desc(n, _ptr(xyz), _ptr(attr), int(attr.shape[1]), int(n_words),
                           int(point_stride), int(index_base))
        h = ctypes.c_void_p()
        check(lib().nrv_create_scene(ctypes.byref(d), ctypes.byref(h)))
        self.h = h
        self.n_words = n_words

    def close(self):
        if self.h:
            lib().nrv_destroy_scene(self.h)
            self.h = None

    __del__ = close


def rasterize(scene: Scene, views, keys, depth=None, mask=None, gattr=None, stream=None):
    """Render + resolve n views; keys[i] uint64/int64 [H,W]; optional planes per view."""
    n = len(views)
    cv = (nrv_view * n)(*[make_view(v) for v in views])
    gb = (nrv_gbuffer * n)()
    for i in range(n):
        gb[i].d_key = _ptr(keys[i])
        gb[i].d_depth = _ptr(depth[i]) if depth else None
        gb[i].d_mask = _ptr(mask[i]) if mask else None
        gb[i].d_attr = _ptr(gattr[i]) if gattr else None
    check(lib().nrv_rasterize(scene.h, cv, n, gb, _stream(stream)))


def pack(depth, mask, gattr, height, width, desc: nrv_pack_desc, prec: int, netin,
         in_scale_inv: float = 1.0, stream=None):
    gb = nrv_gbuffer(None, _ptr(depth), _ptr(mask), _ptr(gattr))
    check(lib().nrv_pack(ctypes.byref(gb), height, width, ctypes.byref(desc), prec,
                         in_scale_inv, _ptr(netin), _stream(stream)))


def resolve(scene: Scene, view, key, depth=None, mask=None, gattr=None, stream=None):
    """Resolve planes from a key image; winners outside the scene's index range read as empty."""
    cv = make_view(view)
    gb = nrv_gbuffer(None, _ptr(depth), _ptr(mask), _ptr(gattr))
    check(lib().nrv_resolve(scene.h, ctypes.byref(cv), _ptr(key), ctypes.byref(gb), _stream(stream)))


def keys_flip_sign(key, stream=None):
    """Flip bit 63 of every key in place: unsigned key order becomes signed int64 order."""
    check(lib().nrv_keys_flip_sign(_ptr(key), key.numel(), _stream(stream)))


def resolve_pack(scene: Scene, view, key, desc: nrv_pack_desc, prec: int, netin,
                 in_scale_inv: float = 1.0, stream=None):
    """Resolve one view's key image straight into the network input (derived channels allowed)."""
    cv = make_view(view)
    check(lib().nrv_resolve_pack(scene.h, ctypes.byref(cv), _ptr(key), ctypes.byref(desc), prec,
                                 in_scale_inv, _ptr(netin), _stream(stream)))


def param_count(c_in: int) -> int:
    n = ctypes.c_int64()
    check(lib().nrv_net_param_count(c_in, ctypes.byref(n)))
    return n.value


def layer_table(c_in: int):
    out = []
    for l in range(lib().nrv_net_num_layers()):
        li = nrv_layer_info()
        check(lib().nrv_net_layer(c_in, l, ctypes.byref(li)))
        out.append((li.name.decode(), li.kind, li.c_in, li.c_out, li.weight_offset, li.bias_offset))
    return out


class Net:
    def __init__(self, c_in: int):
        h = ctypes.c_void_p()
        check(lib().nrv_create_net(c_in, ctypes.byref(h)))
        self.h, self.c_in = h, c_in

    def set_params(self, params, stream=None):
        check(lib().nrv_net_set_params(self.h, _ptr(params), _stream(stream)))

    def init_params(self, seed, params, stream=None):
        """Seeded Xavier-uniform draw into `params` (device float32, param_count), then loaded."""
        check(lib().nrv_net_init_params(self.h, int(seed), _ptr(params), _stream(stream)))

    def get_params(self, out, stream=None):
        check(lib().nrv_net_get_params(self.h, _ptr(out), _stream(stream)))

    def save(self, path, stream=None):
        check(lib().nrv_net_save(self.h, str(path).encode(), _stream(stream)))

    def load(self, path, stream=None):
        check(lib().nrv_net_load(self.h, str(path).encode(), _stream(stream)))

    def set_act_scales(self, scales):
        arr = (F * len(scales))(*[float(s) for s in scales])
        check(lib().nrv_net_set_act_scales(self.h, arr, len(scales), _stream(None)))

    def act_scales(self):
        arr = (F * 21)()
        check(lib().nrv_net_get_act_scales(self.h, arr, 21))
        return [arr[i] for i in range(21)]

    def calibrate(self, netin_bf16, n, height, width, stream=None):
        check(lib().nrv_net_calibrate(self.h, _ptr(netin_bf16), n, height, width, _stream(stream)))

    def shade(self, netin, n, height, width, prec, rgb, stream=None):
        check(lib().nrv_shade(self.h, _ptr(netin), n, height, width, prec, _ptr(rgb), _stream(stream)))

    def backends(self):
        """Per layer: 0 SIMT, 1 tensor cores, -1 not run (most recent forward)."""
        return [lib().nrv_net_layer_backend(self.h, l) for l in range(lib().nrv_net_num_layers())]

    def forward_train(self, netin, n, height, width, prec, rgb, stream=None):
        check(lib().nrv_net_forward_train(self.h, _ptr(netin), n, height, width, prec, _ptr(rgb),
                                          _stream(stream)))

    def layer_wgrad(self, layer, dy, x1, x2, n, height, width, prec, grad, stream=None):
        """Weight and bias gradient of 3x3 layer `layer` into its place in `grad`."""
        check(lib().nrv_net_layer_wgrad(self.h, layer, _ptr(dy), _ptr(x1),
                                        None if x2 is None else _ptr(x2), n, height, width, prec,
                                        _ptr(grad), _stream(stream)))

    def layer_dgrad(self, layer, dy, mask, n, height, width, prec, dx, stream=None):
        """Data gradient of 3x3 layer `layer`, zeroed where `mask` <= 0 (if given)."""
        check(lib().nrv_net_layer_dgrad(self.h, layer, _ptr(dy), None if mask is None else _ptr(mask),
                                        n, height, width, prec, _ptr(dx), _stream(stream)))

    def set_loss(self, weights):
        """Loss of train_step: weights (l1, l2, tv) of nrv_recon_loss; (1, 0, 0) is L1."""
        wt = nrv_loss_weights(*[float(x) for x in weights])
        check(lib().nrv_net_set_loss(self.h, ctypes.byref(wt)))

    def backward(self, drgb, grad, stream=None):
        check(lib().nrv_net_backward(self.h, _ptr(drgb), _ptr(grad), _stream(stream)))

    def train_step(self, params, grad, m, v, step, lr, netin, target, n, height, width, prec, loss,
                   stream=None):
        check(lib().nrv_train_step(self.h, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr,
                                   _ptr(netin), _ptr(target), n, height, width, prec, _ptr(loss),
                                   _stream(stream)))

    def close(self):
        if self.h:
            lib().nrv_destroy_net(self.h)
            self.h = None

    __del__ = close


class GatedNet:
    """The gated post-processing network (include/nrv.h, nrv_gnet_*): BF16 inference."""

    def __init__(self, c_in: int):
        h = ctypes.c_void_p()
        check(lib().nrv_gnet_create(c_in, ctypes.byref(h)))
        self.h, self.c_in = h, c_in

    @staticmethod
    def param_count(c_in: int) -> int:
        n = ctypes.c_int64()
        check(lib().nrv_gnet_param_count(c_in, ctypes.byref(n)))
        return n.value

    def set_params(self, params, stream=None):
        check(lib().nrv_gnet_set_params(self.h, _ptr(params), _stream(stream)))

    def shade(self, netin, n, height, width, rgb, stream=None):
        check(lib().nrv_gnet_shade(self.h, _ptr(netin), n, height, width, _ptr(rgb), _stream(stream)))

    def run_layer(self, layer, x1, x2, n, height, width, y, stream=None):
        check(lib().nrv_gnet_run_layer(self.h, layer, _ptr(x1), None if x2 is None else _ptr(x2), n,
                                       height, width, _ptr(y), _stream(stream)))

    def close(self):
        if self.h:
            lib().nrv_gnet_destroy(self.h)
            self.h = None

    __del__ = close


def l1_loss(y, t, loss, dy=None, stream=None):
    check(lib().nrv_l1_loss(_ptr(y), _ptr(t), y.numel(), _ptr(loss), _ptr(dy), _stream(stream)))


def recon_loss(y, t, weights, loss, dy=None, stream=None):
    """Eq. 1 without the perceptual term on RGB images y, t [n][h][w][3]; weights (l1, l2, tv)."""
    n, h, w, _ = y.shape
    wt = nrv_loss_weights(*[float(x) for x in weights])
    check(lib().nrv_recon_loss(_ptr(y), _ptr(t), n, h, w, ctypes.byref(wt), _ptr(loss), _ptr(dy),
                               _stream(stream)))


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    check(lib().nrv_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), step, lr, b1, b2, eps,
                              _stream(stream)))


def render_batch(scene: Scene, net: Net, desc: nrv_pack_desc, views, rgbs, prec: int,
                 in_scale_inv: float = 1.0, stream=None):
    n = len(views)
    cv = (nrv_view * n)(*[make_view(v) for v in views])
    outs = (P * n)(*[_ptr(r) for r in rgbs])
    check(lib().nrv_render_batch(scene.h, net.h, ctypes.byref(desc), cv, n, outs, prec,
                                 in_scale_inv, _stream(stream)))


def set_profiling(on: bool):
    check(lib().nrv_set_profiling(1 if on else 0))


def timings():
    arr = (F * 4)()
    k = lib().nrv_get_timings(arr, 4)
    return [arr[i] for i in range(k)]


def tune_load(path):
    check(lib().nrv_tune_load(str(path).encode()))


def tune_save(path):
    check(lib().nrv_tune_save(str(path).encode()))


def sync_status(stream=None):
    check(lib().nrv_sync_status(_stream(stream)))
