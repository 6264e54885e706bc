"""Row-streaming 3x3 convolutions over long runs of rows (Sec. 3.3 network layers), against the
oracle's layer on the same BF16 values.

Tall, narrow inputs give each CTA a run of many output rows, so the TMEM ring of accumulator
blocks wraps (the MMAs split where three blocks straddle the ring's end), several groups are in
flight between the issuer and the two groups of epilogue warps, and runs cross images.  The
bound is the per-layer one of test_gpu_conv: one BF16 unit in the last place plus the FP32
summation error bound, and almost all outputs bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import make_params, torch_dev
from oracle import unet

pytestmark = pytest.mark.gpu


def _bf16(t):
    return oracle.bf16_value(oracle.bf16_bits(np.asarray(t, np.float32))).astype(np.float64)


# (layer name, images, height, width): one 126-pixel tile column, or two
CASES = [("e0b", 1, 4096, 120), ("d0a", 3, 700, 120), ("d1a", 1, 2048, 120), ("e2b", 2, 1024, 250)]


@pytest.mark.parametrize("name,n,h,w", CASES)
def test_long_runs(name, n, h, w):
    import torch
    from paper_2407_19097_gb300 import nrv
    c0 = 5
    names = [l[0] for l in unet.layers(c0)]
    layer = names.index(name)
    flat = make_params(c0, seed=layer + 71, bias_sigma=0.1)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    _, _, ci, co = unet.layers(c0)[layer]
    concat = name in ("d2a", "d1a", "d0a")
    c1 = ci // 2 if concat else ci
    rng = np.random.default_rng(layer + 5)
    x = rng.standard_normal((n, h, w, ci)).astype(np.float32)
    W, b = unet.unflatten(flat.astype(np.float64), c0)[name]
    xt = torch.from_numpy(x).to(torch_dev()).to(torch.bfloat16)
    x1 = xt[..., :c1].contiguous()
    x2 = xt[..., c1:].contiguous() if concat else None
    y = torch.empty((n, h, w, co), dtype=torch.bfloat16, device=torch_dev())
    nrv.check(nrv.lib().nrv_net_run_layer(net.h, layer, nrv._ptr(x1), nrv._ptr(x2), n, h, w, 1,
                                          nrv._ptr(y), nrv._stream()))
    torch.cuda.synchronize()
    assert net.backends()[layer] == 1
    got = y.float().cpu().numpy().astype(np.float64)
    xin = _bf16(x)
    Wq = _bf16(W)
    pre = unet.conv3(xin, Wq, b)
    ref = _bf16(unet.relu(pre))
    S = unet.conv3(np.abs(xin), np.abs(Wq), np.abs(b))
    K = 9 * ci
    # a ReLU decision within FP32 accumulation error of zero is not compared
    ok = ~(np.abs(pre) <= 1e-5 * np.abs(pre).max())
    exact = np.mean(got[ok] == ref[ok])
    big = np.maximum(np.abs(got), np.abs(ref))[ok]
    ulp = np.exp2(np.floor(np.log2(np.maximum(big, 1e-30))) - 7)
    bound = ulp + K * 2.0 ** -24 / (1 - K * 2.0 ** -24) * S[ok]
    worst = float(np.max(np.abs(got[ok] - ref[ok]) / bound))
    assert exact >= 0.99 and worst <= 1.0, (exact, worst)


# gated layers (Sec. 3.3's gated network): (layer name, images, height, width)
GATED_CASES = [("e0", 1, 4096, 120), ("d1", 2, 1024, 120)]


@pytest.mark.parametrize("name,n,h,w", GATED_CASES)
def test_gated_long_runs(name, n, h, w):
    import torch
    from paper_2407_19097_gb300 import nrv
    from oracle import gated
    from test_gpu_gated import _dev_bf16, _kernel_params, _params
    c0 = 5
    names = [l[0] for l in gated.layers(c0)]
    layer = names.index(name)
    flat = _params(c0, seed=layer + 41)
    net = nrv.GatedNet(c0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    P = _kernel_params(flat, c0)
    _, _, cin, cout = gated.layers(c0)[layer]
    rng = np.random.default_rng(layer + 9)
    if name == "e0":
        x1 = np.zeros((n, h, w, 8), np.float32)
        x1[..., :c0] = rng.standard_normal((n, h, w, c0))
        x2 = None
        xin = _bf16(x1)[..., :c0]
    else:
        x1 = rng.standard_normal((n, h, w, cin // 2)).astype(np.float32)
        x2 = rng.standard_normal((n, h, w, cin // 2)).astype(np.float32)
        xin = np.concatenate([_bf16(x1), _bf16(x2)], -1)
    y = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device=torch_dev())
    net.run_layer(layer, _dev_bf16(x1), None if x2 is None else _dev_bf16(x2), n, h, w, y)
    ref = gated.gated(xin, *P[name])
    torch.cuda.synchronize()
    got = y.float().cpu().numpy().astype(np.float64)
    # BF16 output rounding (half an ulp, 2^-9 relative) plus FP32 accumulation
    scale = float(np.sqrt(np.mean(ref * ref)))
    err = np.abs(got - ref) / (np.abs(ref) * 2.0 ** -8 + 2e-4 * scale + 1e-6)
    assert err.max() <= 1.0, (name, float(err.max()))
