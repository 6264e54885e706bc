"""CPU ORACLE (test infrastructure only): the fixed post-processing U-Net in float64.

Only tests, the smoke check and the benchmark's CPU-baseline leg use this module;
the rendering library never does, and nothing here is shared with it.

The paper's post-processing network is a U-Net (Sec. 3.3): an encoder with four
downsampling stages and 2x2 average pooling, a decoder that upsamples with
transposed convolutions and fuses skip connections.  The network built here is
the fixed plain variant of it: four levels with 16/32/64/128 channels, two 3x3
"same" convolutions + bias + ReLU per level, 2x2 average pooling between encoder
levels, a 2x2 stride-2 transposed convolution (bias, no activation) per decoder
level, concatenation [upsampled, skip], and a linear 1x1 head to RGB.  Tensors
are NHWC, float64.

Conventions (PyTorch's): convolution is cross-correlation with zero padding,
conv weights are (C_out, C_in, 3, 3), transposed-conv weights (C_in, C_out, 2, 2)
with y[2i+a, 2j+b, o] = b[o] + sum_c x[i, j, c] * W[c, o, a, b], head weights
(C_out, C_in).  The flat parameter vector stores, layer by layer in LAYERS order,
the weight in that layout and then the bias.

Each step is its textbook definition, with numpy matmul as the only library
primitive; the backward is the analytic gradient of the same steps.
"""
from __future__ import annotations

import numpy as np

# (name, kind, c_in, c_out); c_in of the first layer is the network input width.
def layers(c0: int):
    return [
        ("e0a", "conv3", c0, 16), ("e0b", "conv3", 16, 16),
        ("e1a", "conv3", 16, 32), ("e1b", "conv3", 32, 32),
        ("e2a", "conv3", 32, 64), ("e2b", "conv3", 64, 64),
        ("e3a", "conv3", 64, 128), ("e3b", "conv3", 128, 128),
        ("up3", "convT2", 128, 64), ("d2a", "conv3", 128, 64), ("d2b", "conv3", 64, 64),
        ("up2", "convT2", 64, 32), ("d1a", "conv3", 64, 32), ("d1b", "conv3", 32, 32),
        ("up1", "convT2", 32, 16), ("d0a", "conv3", 32, 16), ("d0b", "conv3", 16, 16),
        ("head", "conv1", 16, 3),
    ]


def weight_shape(kind: str, cin: int, cout: int):
    return {"conv3": (cout, cin, 3, 3), "convT2": (cin, cout, 2, 2), "conv1": (cout, cin)}[kind]


def fans(kind: str, cin: int, cout: int):
    """Xavier fans: C_in*k^2 and C_out*k^2 for every layer, transposed ones included."""
    k2 = {"conv3": 9, "convT2": 4, "conv1": 1}[kind]
    return cin * k2, cout * k2


def param_count(c0: int) -> int:
    return sum(int(np.prod(weight_shape(k, ci, co))) + co for _, k, ci, co in layers(c0))


def unflatten(flat: np.ndarray, c0: int) -> dict:
    """Flat float vector -> {name: (W, b)} views in float64."""
    flat = np.asarray(flat, np.float64)
    out, o = {}, 0
    for name, kind, ci, co in layers(c0):
        shp = weight_shape(kind, ci, co)
        n = int(np.prod(shp))
        out[name] = (flat[o:o + n].reshape(shp), flat[o + n:o + n + co])
        o += n + co
    assert o == flat.size, (o, flat.size)
    return out


def flatten(grads: dict, c0: int) -> np.ndarray:
    parts = []
    for name, _, _, _ in layers(c0):
        w, b = grads[name]
        parts += [np.asarray(w, np.float64).reshape(-1), np.asarray(b, np.float64).reshape(-1)]
    return np.concatenate(parts)


# ----------------------------------------------------------------------------- forward ops

def conv3(x, w, b):
    """y[n,i,j,o] = b[o] + sum_{c,u,v} w[o,c,u,v] * x[n, i+u-1, j+v-1, c], zero outside."""
    n, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (n, h, wd, w.shape[0])).copy()
    for u in range(3):
        for v in range(3):
            y += xp[:, u:u + h, v:v + wd, :] @ w[:, :, u, v].T
    return y


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    """Mean of each 2x2 window, stride 2."""
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 0::2] + x[:, 1::2, 1::2])


def convT2(x, w, b):
    """y[n, 2i+a, 2j+c, o] = b[o] + sum_k x[n,i,j,k] * w[k,o,a,c]."""
    n, h, wd, _ = x.shape
    y = np.empty((n, 2 * h, 2 * wd, w.shape[1]))
    for a in range(2):
        for c in range(2):
            y[:, a::2, c::2, :] = x @ w[:, :, a, c] + b
    return y


def conv1(x, w, b):
    return x @ w.T + b


# ----------------------------------------------------------------------------- network

def forward(x, params: dict, save: bool = False, q=None):
    """U-Net forward on NHWC float64 input with H, W divisible by 8.  Returns RGB (and the
    saved activations when save=True; "pre:<layer>" holds each ReLU layer's pre-activation).

    q, if given, is applied to every tensor the network stores between layers (the input,
    each ReLU output, pooled and upsampled tensors), e.g. rounding to the storage precision
    of a reduced-precision network; the head's output is not rounded."""
    rq = (lambda t: t) if q is None else q
    x = rq(np.asarray(x, np.float64))
    s = {"x": x}

    def cr(name, inp):
        w, b = params[name]
        pre = conv3(inp, w, b)
        y = rq(relu(pre))
        s[name] = y
        if save:
            s["pre:" + name] = pre
        return y

    a = cr("e0b", cr("e0a", x))
    p = rq(avgpool2(a)); s["p0"] = p
    a = cr("e1b", cr("e1a", p))
    p = rq(avgpool2(a)); s["p1"] = p
    a = cr("e2b", cr("e2a", p))
    p = rq(avgpool2(a)); s["p2"] = p
    a = cr("e3b", cr("e3a", p))
    for up, da, db, skip in (("up3", "d2a", "d2b", "e2b"), ("up2", "d1a", "d1b", "e1b"),
                             ("up1", "d0a", "d0b", "e0b")):
        u = rq(convT2(a, *params[up])); s[up] = u
        c = np.concatenate([u, s[skip]], axis=-1); s["cat" + up] = c
        a = cr(db, cr(da, c))
    y = conv1(a, *params["head"])
    return (y, s) if save else y


def relu_margin(s: dict) -> float:
    """Smallest |pre-activation| over every ReLU layer, relative to the largest: a ReLU
    decision closer to zero than rounding can flip between two precisions."""
    pres = [v for k, v in s.items() if k.startswith("pre:")]
    lo = min(float(np.abs(v).min()) for v in pres)
    hi = max(float(np.abs(v).max()) for v in pres)
    return lo / hi


# ----------------------------------------------------------------------------- backward ops

def conv3_bwd(x, w, dy):
    """Gradients of conv3 w.r.t. x, w, b given dL/dy."""
    n, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    d2 = dy.reshape(-1, dy.shape[-1])
    for u in range(3):
        for v in range(3):
            xs = xp[:, u:u + h, v:v + wd, :].reshape(-1, x.shape[-1])
            dw[:, :, u, v] = d2.T @ xs
            dxp[:, u:u + h, v:v + wd, :] += dy @ w[:, :, u, v]
    return dxp[:, 1:-1, 1:-1, :], dw, d2.sum(axis=0)


def avgpool2_bwd(dy):
    n, h, w, c = dy.shape
    dx = np.empty((n, 2 * h, 2 * w, c))
    for a in range(2):
        for b in range(2):
            dx[:, a::2, b::2] = 0.25 * dy
    return dx


def convT2_bwd(x, w, dy):
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    xs = x.reshape(-1, x.shape[-1])
    for a in range(2):
        for c in range(2):
            g = dy[:, a::2, c::2, :]
            dw[:, :, a, c] = xs.T @ g.reshape(-1, g.shape[-1])
            dx += g @ w[:, :, a, c].T
    return dx, dw, dy.reshape(-1, dy.shape[-1]).sum(axis=0)


def backward(dy, params: dict, s: dict, q=None):
    """Analytic gradients of the network w.r.t. its parameters and its input, given dL/dRGB and
    the saved forward activations.  ReLU'(0) = 0.  q, if given, is applied to every gradient
    tensor passed between layers (the same storage rounding as in forward); parameter
    gradients are not rounded."""
    rq = (lambda t: t) if q is None else q
    g = {}
    wh, _ = params["head"]
    a_last = s["d0b"]
    d2 = dy.reshape(-1, dy.shape[-1])
    g["head"] = (d2.T @ a_last.reshape(-1, a_last.shape[-1]), d2.sum(axis=0))
    da = rq(dy @ wh)

    def cr_bwd(name, inp, dout):
        dout = dout * (s[name] > 0)
        dx, dw, db = conv3_bwd(inp, params[name][0], dout)
        g[name] = (dw, db)
        return rq(dx)

    dskip = {}
    # decoder, finest level first; `below` is the activation the transposed conv upsampled
    for up, da_name, db_name, skip, below in (("up1", "d0a", "d0b", "e0b", "d1b"),
                                              ("up2", "d1a", "d1b", "e1b", "d2b"),
                                              ("up3", "d2a", "d2b", "e2b", "e3b")):
        d = cr_bwd(db_name, s[da_name], da)
        dc = cr_bwd(da_name, s["cat" + up], d)
        cu = s[up].shape[-1]
        dskip[skip] = dc[..., cu:]
        dx, dw, db = convT2_bwd(s[below], params[up][0], dc[..., :cu])
        g[up] = (dw, db)
        da = rq(dx)
    # encoder, deepest first
    d = cr_bwd("e3b", s["e3a"], da)
    d = cr_bwd("e3a", s["p2"], d)
    for ea, eb, pin in (("e2a", "e2b", "p1"), ("e1a", "e1b", "p0"), ("e0a", "e0b", "x")):
        d = rq(avgpool2_bwd(d) + dskip[eb])
        d = cr_bwd(eb, s[ea], d)
        d = cr_bwd(ea, s[pin], d)
    return g, d


# ----------------------------------------------------------------------------- training

def l1_loss(y, t):
    """mean |y - t| and its gradient sign(y - t) / numel, sign(0) = 0."""
    diff = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.abs(diff).mean()), np.sign(diff) / diff.size


def recon_tv_loss(y, t, l1=0.0, l2=0.0, tv=0.0):
    """Eq. (1) without its perceptual term, on RGB images y, t [n, h, w, 3]:
    l1 mean|y - t| + l2 mean (y - t)^2 (the pixel-wise reconstruction term) + tv times the 2-D
    total variation of y (mean |y[:, :, x+1] - y[:, :, x]| over horizontal pairs plus
    mean |y[:, y+1] - y[:, y]| over vertical pairs).  Returns (loss, dL/dy), sign(0) = 0."""
    y = np.asarray(y, np.float64)
    d = y - np.asarray(t, np.float64)
    loss = l1 * np.abs(d).mean() + l2 * (d * d).mean()
    g = l1 * np.sign(d) / d.size + 2.0 * l2 * d / d.size
    if tv != 0.0:
        dh = y[:, :, 1:] - y[:, :, :-1]
        dv = y[:, 1:] - y[:, :-1]
        if dh.size:
            loss += tv * np.abs(dh).mean()
            sh = np.sign(dh) / dh.size
            g[:, :, 1:] += tv * sh
            g[:, :, :-1] -= tv * sh
        if dv.size:
            loss += tv * np.abs(dv).mean()
            sv = np.sign(dv) / dv.size
            g[:, 1:] += tv * sv
            g[:, :-1] -= tv * sv
    return float(loss), g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), step t >= 1, no weight decay; returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
