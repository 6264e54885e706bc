"""Per-layer GPU parity of the U-Net's convolutions (Sec. 3.3 network): every 3x3 and every
2x2 stride-2 transposed convolution run alone through nrv_net_run_layer on seeded inputs,
against the oracle's layer on the same values.

BF16 (tensor cores): inputs and weights are BF16 on both sides, the oracle accumulates in
float64 and rounds the output to BF16 once; the GPU accumulates in FP32.  Outputs must agree
within one BF16 unit in the last place plus the FP32 summation error bound, and almost all bit
for bit.  FP32 (SIMT): within 1e-5 relative of the float64 oracle.  Shapes cover several
128-pixel tiles with a ragged last tile, two images, the 8-channel first layer and the
concatenating decoder layers."""
import numpy as np
import pytest

import oracle
from gpu_util import make_params, torch_dev
from oracle import unet

pytestmark = pytest.mark.gpu


def _bf16(t):
    return oracle.bf16_value(oracle.bf16_bits(np.asarray(t, np.float32))).astype(np.float64)


LAYERS = [(i, name, kind) for i, (name, kind, _, _) in enumerate(unet.layers(5)) if kind != "conv1"]


def _run(net, layer, x1, x2, n, h, w, prec, y):
    from paper_2407_19097_gb300 import nrv
    nrv.check(nrv.lib().nrv_net_run_layer(net.h, layer, nrv._ptr(x1), nrv._ptr(x2), n, h, w, prec,
                                          nrv._ptr(y), nrv._stream()))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layer,name,kind", LAYERS)
def test_layer(layer, name, kind, prec):
    import torch
    from paper_2407_19097_gb300 import nrv
    c0 = 5
    flat = make_params(c0, seed=layer + 31, bias_sigma=0.1)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    _, _, ci, co = unet.layers(c0)[layer]
    cin = 8 if layer == 0 else ci
    concat = name in ("d2a", "d1a", "d0a")
    c1 = cin // 2 if concat else cin
    n, h, w = 2, 5, 300                     # 3 tiles of 128 pixels per row, the last ragged
    rng = np.random.default_rng(layer)
    x = rng.standard_normal((n, h, w, cin)).astype(np.float32)
    if layer == 0:
        x[..., c0:] = 0.0                   # padding channels of the packed input
    W, b = unet.unflatten(flat.astype(np.float64), c0)[name]
    dt = torch.bfloat16 if prec == 1 else torch.float32
    xt = torch.from_numpy(x).to(torch_dev()).to(dt)
    x1 = xt[..., :c1].contiguous()
    x2 = xt[..., c1:].contiguous() if concat else None
    oh, ow = (h, w) if kind == "conv3" else (2 * h, 2 * w)
    y = torch.empty((n, oh, ow, co), dtype=dt, device=torch_dev())
    _run(net, layer, x1, x2, n, h, w, prec, y)
    torch.cuda.synchronize()
    got = y.float().cpu().numpy().astype(np.float64)
    xin = (_bf16(x) if prec == 1 else x.astype(np.float64))[..., :ci]
    Wq = _bf16(W) if prec == 1 else W
    if kind == "conv3":
        pre = unet.conv3(xin, Wq, b)
        out = unet.relu(pre)
        S = unet.conv3(np.abs(xin), np.abs(Wq), np.abs(b))
        K = 9 * ci
    else:
        pre = unet.convT2(xin, Wq, b)
        out = pre
        S = unet.convT2(np.abs(xin), np.abs(Wq), np.abs(b))
        K = ci
    if prec == 1:
        assert net.backends()[layer] == 1
        ref = _bf16(out)
        # a ReLU decision within FP32 accumulation error of zero is not compared
        amb = (np.abs(pre) <= 1e-5 * np.abs(pre).max()) if kind == "conv3" else np.zeros(pre.shape, bool)
        assert amb.mean() < 1e-3
        ok = ~amb
        exact = np.mean(got[ok] == ref[ok])
        # |got - ref| <= one BF16 ulp of the larger value + gamma_K * sum|w x| (FP32 summation
        # error bound over K products, u = 2^-24)
        big = np.maximum(np.abs(got), np.abs(ref))[ok]
        ulp = np.exp2(np.floor(np.log2(np.maximum(big, 1e-30))) - 7)
        bound = ulp + K * 2.0 ** -24 / (1 - K * 2.0 ** -24) * S[ok]
        worst = float(np.max(np.abs(got[ok] - ref[ok]) / bound))
        assert exact >= 0.99 and worst <= 1.0, (exact, worst)
    else:
        err = np.abs(got - out).max() / max(1.0, np.abs(out).max())
        assert err <= 1e-5, err
