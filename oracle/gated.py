"""CPU ORACLE (test infrastructure only): the gated post-processing network of Sec. 3.3 in
float64, at reduced width.

The paper's network is a U-Net whose blocks are gated convolutions (Yu et al.) with ELU --
out = ELU(W_f * x + b_f) (.) sigmoid(W_g * x + b_g) -- followed in the encoder by 2x2 average
pooling; a 1x1 convolution of the G-buffers (keeping their channel count) is downscaled by 0.5
per level and concatenated to the first block of every encoder level; the decoder upsamples
with transposed convolutions and concatenates the skip connections.  Built here with four
levels of 16/32/64/128 channels (the paper's progression starts at 64 over five levels):

    g0 = 1x1(x)                       g_l = avgpool(g_{l-1})          (C0 channels)
    e0 = gated(g0)                    e_l = gated([avgpool(e_{l-1}), g_l])   l = 1..3
    u2 = convT(e3)   d2 = gated([u2, e2])
    u1 = convT(d2)   d1 = gated([u1, e1])
    u0 = convT(d1)   d0 = gated([u0, e0])
    rgb = 1x1(d0)

Convolution conventions and the transposed convolution are those of oracle/unet.py; every step
is its definition in numpy (matmul the only library primitive).
"""
from __future__ import annotations

import numpy as np

from .unet import avgpool2, conv1, conv3, convT2

WIDTHS = (16, 32, 64, 128)


def layers(c0: int):
    """(name, kind, c_in, c_out); kind "gated" holds a feature and a gate 3x3 conv."""
    w = WIDTHS
    return [("inj", "conv1", c0, c0),
            ("e0", "gated", c0, w[0]), ("e1", "gated", w[0] + c0, w[1]),
            ("e2", "gated", w[1] + c0, w[2]), ("e3", "gated", w[2] + c0, w[3]),
            ("up2", "convT2", w[3], w[2]), ("d2", "gated", 2 * w[2], w[2]),
            ("up1", "convT2", w[2], w[1]), ("d1", "gated", 2 * w[1], w[1]),
            ("up0", "convT2", w[1], w[0]), ("d0", "gated", 2 * w[0], w[0]),
            ("head", "conv1", w[0], 3)]


def shapes(kind: str, cin: int, cout: int):
    """Flat-vector layout of one layer: the tensors in order."""
    if kind == "gated":
        return [(cout, cin, 3, 3), (cout,), (cout, cin, 3, 3), (cout,)]
    if kind == "convT2":
        return [(cin, cout, 2, 2), (cout,)]
    return [(cout, cin), (cout,)]


def param_count(c0: int) -> int:
    return sum(int(np.prod(s)) for _, k, ci, co in layers(c0) for s in shapes(k, ci, co))


def unflatten(flat, c0: int) -> dict:
    flat = np.asarray(flat, np.float64)
    out, o = {}, 0
    for name, kind, ci, co in layers(c0):
        ts = []
        for s in shapes(kind, ci, co):
            n = int(np.prod(s))
            ts.append(flat[o:o + n].reshape(s))
            o += n
        out[name] = tuple(ts)
    assert o == flat.size, (o, flat.size)
    return out


def elu(x):
    return np.where(x > 0.0, x, np.expm1(np.minimum(x, 0.0)))


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def gated(x, wf, bf, wg, bg):
    """ELU(conv3(x; W_f) + b_f) * sigmoid(conv3(x; W_g) + b_g)."""
    return elu(conv3(x, wf, bf)) * sigmoid(conv3(x, wg, bg))


def forward(x, params: dict, q=None):
    """Gated network on NHWC float64 input (H, W divisible by 8).  q, if given, rounds every
    tensor the network stores (input, injected pyramid, block outputs, pooled and upsampled
    tensors) to a storage precision; the RGB output is not rounded."""
    rq = (lambda t: t) if q is None else q
    x = rq(np.asarray(x, np.float64))
    cat = lambda a, b: np.concatenate([a, b], axis=-1)
    g = [rq(conv1(x, *params["inj"]))]
    for _ in range(3):
        g.append(rq(avgpool2(g[-1])))
    e = [rq(gated(g[0], *params["e0"]))]
    for l in range(1, 4):
        e.append(rq(gated(cat(rq(avgpool2(e[l - 1])), g[l]), *params["e%d" % l])))
    d = e[3]
    for l in (2, 1, 0):
        u = rq(convT2(d, *params["up%d" % l]))
        d = rq(gated(cat(u, e[l]), *params["d%d" % l]))
    return conv1(d, *params["head"])
