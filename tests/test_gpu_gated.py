"""The gated post-processing network (Sec. 3.3's form) on the tensor cores against the float64
oracle: every layer alone on the same BF16 inputs (3x3 and transposed-conv weights rounded to
BF16 on both sides, as the kernels use them), and the whole network -- one image and a batch --
at PSNR >= 45 dB over the oracle's output range and max abs <= 2e-2."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import psnr_range, torch_dev
from oracle import gated
from oracle.unet import avgpool2, conv1, convT2

pytestmark = pytest.mark.gpu


def _params(c0, seed=3, bias_sigma=0.05):
    flat = []
    for t, (name, kind, ci, co) in enumerate(gated.layers(c0)):
        for k, shp in enumerate(gated.shapes(kind, ci, co)):
            if len(shp) == 1:
                flat.append((bias_sigma * I.normal_array(seed, 3000 + 8 * t + k, shp[0])).astype(np.float32))
            else:
                k2 = 9 if kind == "gated" else (4 if kind == "convT2" else 1)
                flat.append(I.xavier_uniform(seed, 2000 + 8 * t + k, shp, ci * k2, co * k2).ravel())
    return np.concatenate(flat).astype(np.float32)


def _bf16(a):
    return oracle.bf16_value(oracle.bf16_bits(np.asarray(a, np.float32))).astype(np.float64)


def _kernel_params(flat, c0):
    """The weights as the kernels use them: 3x3 and transposed-conv weights in BF16, the 1x1
    layers and every bias in FP32."""
    P = gated.unflatten(flat, c0)
    out = {}
    for name, kind, _, _ in gated.layers(c0):
        t = P[name]
        if kind == "gated":
            out[name] = (_bf16(t[0]), t[1], _bf16(t[2]), t[3])
        elif kind == "convT2":
            out[name] = (_bf16(t[0]), t[1])
        else:
            out[name] = t
    return out


def _input(n, h, w, c0, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, h, w, 8), np.float32)
    cov = rng.uniform(0, 1, (n, h, w)) < 0.6
    x[..., :c0 - 2] = rng.standard_normal((n, h, w, c0 - 2))
    x[..., c0 - 2] = rng.uniform(0, 1, (n, h, w))
    x[..., c0 - 1] = 1.0
    x[~cov] = 0.0
    return x


def _dev_bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch_dev()).to(torch.bfloat16)


LAYERS = [(i, n) for i, (n, k, _, _) in enumerate(gated.layers(5)) if n != "head"]


@pytest.mark.parametrize("layer,name", LAYERS)
def test_gated_layer(layer, name):
    import torch
    from paper_2407_19097_gb300 import nrv
    c0 = 5
    flat = _params(c0, seed=layer + 11)
    net = nrv.GatedNet(c0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    P = _kernel_params(flat, c0)
    kind = gated.layers(c0)[layer][1]
    cin, cout = gated.layers(c0)[layer][2:]
    n, h, w = 2, 22, 270                    # several 126-pixel tiles and a ragged one
    rng = np.random.default_rng(layer)
    if name == "inj":
        x1 = _input(n, h, w, c0, layer)
        x2 = None
        xin = _bf16(x1)[..., :c0]
    elif name == "e0":
        x1 = np.zeros((n, h, w, 8), np.float32)
        x1[..., :c0] = rng.standard_normal((n, h, w, c0))
        x2 = None
        xin = _bf16(x1)[..., :c0]
    elif name in ("e1", "e2", "e3"):
        x1 = np.maximum(rng.standard_normal((n, h, w, cin - c0)), -0.5).astype(np.float32)
        x2 = np.zeros((n, h, w, 8), np.float32)
        x2[..., :c0] = rng.standard_normal((n, h, w, c0))
        xin = np.concatenate([_bf16(x1), _bf16(x2)[..., :c0]], -1)
    elif kind == "convT2":
        x1 = rng.standard_normal((n, h, w, cin)).astype(np.float32)
        x2 = None
        xin = _bf16(x1)
    else:
        x1 = rng.standard_normal((n, h, w, cin // 2)).astype(np.float32)
        x2 = rng.standard_normal((n, h, w, cin // 2)).astype(np.float32)
        xin = np.concatenate([_bf16(x1), _bf16(x2)], -1)
    oh, ow = (2 * h, 2 * w) if kind == "convT2" else (h, w)
    oc = 8 if name == "inj" else cout
    y = torch.empty((n, oh, ow, oc), dtype=torch.bfloat16, device=torch_dev())
    net.run_layer(layer, _dev_bf16(x1), None if x2 is None else _dev_bf16(x2), n, h, w, y)
    if name == "inj":
        ref = conv1(xin, *P["inj"])
    elif kind == "gated":
        ref = gated.gated(xin, *P[name])
    else:
        ref = convT2(xin, *P[name])
    torch.cuda.synchronize()
    got = y.float().cpu().numpy().astype(np.float64)[..., :ref.shape[-1]]
    if name == "inj":
        assert np.all(y.float().cpu().numpy()[..., c0:] == 0)
    # BF16 output rounding (half an ulp, 2^-9 relative) plus FP32 accumulation
    scale = float(np.sqrt(np.mean(ref * ref)))
    err = np.abs(got - ref) / (np.abs(ref) * 2.0 ** -8 + 2e-4 * scale + 1e-6)
    assert err.max() <= 1.0, (name, float(err.max()))


@pytest.mark.parametrize("c0,n,h,w", [(5, 1, 120, 200), (7, 2, 64, 136)])
def test_gated_network_vs_fp64(c0, n, h, w):
    import torch
    from paper_2407_19097_gb300 import nrv
    flat = _params(c0, seed=c0)
    net = nrv.GatedNet(c0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    x = _input(n, h, w, c0, seed=2)
    rgb = torch.empty((n, h, w, 3), device=torch_dev())
    net.shade(_dev_bf16(x), n, h, w, rgb)
    ref = gated.forward(_bf16(x)[..., :c0], gated.unflatten(flat, c0))
    torch.cuda.synchronize()
    got = rgb.cpu().numpy()
    p, err = psnr_range(got, ref), float(np.abs(got - ref).max())
    print(f"gated network BF16 vs float64: {p:.1f} dB, max abs {err:.2e}")
    assert p >= 45.0 and err <= 2e-2, (p, err)
