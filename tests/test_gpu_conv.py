"""Per-layer GPU parity of the 3x3 convolution (Sec. 3.3 network): every conv layer of the
U-Net run alone through nrv_net_conv3 on seeded inputs, against the oracle's convolution on
the same values.

BF16 (tensor cores): inputs and weights are BF16 on both sides, the oracle accumulates in
float64 and rounds the ReLU output to BF16 once; the GPU accumulates in FP32.  Outputs must
agree to one BF16 unit in the last place, and almost all bit for bit.
FP32 (SIMT): within 1e-5 relative of the float64 oracle.
Shapes cover several 128-pixel tiles with a ragged last tile, more than one image, the
8-channel first layer and the concatenating decoder layers."""
import numpy as np
import pytest

import oracle
from gpu_util import make_params, torch_dev
from oracle import unet

pytestmark = pytest.mark.gpu


def _bf16(t):
    return oracle.bf16_value(oracle.bf16_bits(np.asarray(t, np.float32))).astype(np.float64)


CONV_LAYERS = [(i, name) for i, (name, kind, _, _) in enumerate(unet.layers(5)) if kind == "conv3"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layer,name", CONV_LAYERS)
def test_conv_layer(layer, name, prec):
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
    y = torch.empty((n, h, w, co), dtype=dt, device=torch_dev())
    nrv.check(nrv.lib().nrv_net_conv3(net.h, layer, nrv._ptr(x1), nrv._ptr(x2), n, h, w, prec,
                                      nrv._ptr(y), nrv._stream()))
    torch.cuda.synchronize()
    got = y.float().cpu().numpy().astype(np.float64)
    if prec == 1:
        assert net.backends()[layer] == 1
        xin = _bf16(x)[..., :ci]
        pre = unet.conv3(xin, _bf16(W), b)
        ref = _bf16(unet.relu(pre))
        # a ReLU decision within FP32 accumulation error of zero is not compared
        amb = np.abs(pre) <= 1e-5 * np.abs(pre).max()
        assert amb.mean() < 1e-3
        ok = ~amb
        exact = np.mean(got[ok] == ref[ok])
        # |got - ref| <= one BF16 ulp of the larger value + gamma_K * sum|w x| (FP32 summation
        # error bound over K = 9 * C_in products, u = 2^-24)
        big = np.maximum(np.abs(got), np.abs(ref))[ok]
        ulp = np.exp2(np.floor(np.log2(np.maximum(big, 1e-30))) - 7)
        K = 9 * ci
        S = unet.conv3(np.abs(xin), np.abs(_bf16(W)), np.abs(b))[ok]
        bound = ulp + K * 2.0 ** -24 / (1 - K * 2.0 ** -24) * S
        worst = float(np.max(np.abs(got[ok] - ref[ok]) / bound))
        assert exact >= 0.99 and worst <= 1.0, (exact, worst)
    else:
        ref = unet.relu(unet.conv3(x[..., :ci].astype(np.float64), W, b))
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err <= 1e-5, err
