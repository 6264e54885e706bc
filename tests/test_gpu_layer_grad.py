"""Per-layer GPU parity of the backward pass of the U-Net's 3x3 convolutions (Sec. 3.3
network): weight and bias gradients through nrv_net_layer_wgrad and data gradients through
nrv_net_layer_dgrad, run one layer at a time, against the oracle's conv3_bwd on the same values.

Weight gradients:

BF16 (tensor cores): the output gradient and the input are BF16 values on both sides; every
product of two BF16 values is exact in FP32, so the only difference is the summation: the GPU
sums in FP32 (per MMA, per 128-pixel tile, per K-split, then the splits in a fixed order), the
oracle in float64.  The bound is the FP32 summation error of a sum of |terms|:
|got - ref| <= 1e-5 * sum_p |dy * x| per weight, plus 1e-30.  FP32 (CUDA cores): the same bound.
Shapes: three 128-pixel tiles per row with a ragged last one, two images and enough rows that
every K-split of the tensor-core kernel sums several tiles; the concatenating decoder layers
take two inputs; the first layer reads the 8-channel packed input (CUDA cores in both
precisions: 8 channels are less than one 16-channel group)."""
import numpy as np
import pytest

import oracle
from gpu_util import make_params, torch_dev
from oracle import unet

pytestmark = pytest.mark.gpu


def _bf16(t):
    return oracle.bf16_value(oracle.bf16_bits(np.asarray(t, np.float32))).astype(np.float64)


C0 = 5
CONV3 = [(i, name) for i, (name, kind, _, _) in enumerate(unet.layers(C0)) if kind == "conv3"]


def _offsets(c0):
    off, o = {}, 0
    for name, kind, ci, co in unet.layers(c0):
        wsz = int(np.prod(unet.weight_shape(kind, ci, co)))
        off[name] = (o, wsz, o + wsz, co)
        o += wsz + co
    return off, o


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layer,name", CONV3)
def test_layer_wgrad(layer, name, prec):
    import torch
    from paper_2407_19097_gb300 import nrv
    net = nrv.Net(C0)
    net.set_params(torch.from_numpy(make_params(C0, seed=7)).to(torch_dev()))
    _, _, ci, co = unet.layers(C0)[layer]
    cin = 8 if layer == 0 else ci
    concat = name in ("d2a", "d1a", "d0a")
    c1 = cin // 2 if concat else cin
    # enough rows that each K-split sums several tiles (up to 304 splits for 16 channels in)
    n, h, w = 2, 200 if co <= 32 else 120, 300
    rng = np.random.default_rng(100 + layer)
    x = rng.standard_normal((n, h, w, cin)).astype(np.float32)
    dy = (rng.standard_normal((n, h, w, co)) * 0.1).astype(np.float32)
    if layer == 0:
        x[..., C0:] = 0.0
    dt = torch.bfloat16 if prec == 1 else torch.float32
    xt = torch.from_numpy(x).to(torch_dev()).to(dt)
    dyt = torch.from_numpy(dy).to(torch_dev()).to(dt).contiguous()
    x1 = xt[..., :c1].contiguous()
    x2 = xt[..., c1:].contiguous() if concat else None
    off, total = _offsets(C0)
    grad = torch.full((total,), float("nan"), device=torch_dev())
    net.layer_wgrad(layer, dyt, x1, x2, n, h, w, prec, grad)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    xv = _bf16(x) if prec == 1 else x.astype(np.float64)
    dv = _bf16(dy) if prec == 1 else dy.astype(np.float64)
    xr = xv[..., :ci]                                   # the layer's real input channels
    wz = np.zeros(unet.weight_shape("conv3", ci, co))
    _, dw_ref, db_ref = unet.conv3_bwd(xr, wz, dv)
    _, dw_abs, db_abs = unet.conv3_bwd(np.abs(xr), wz, np.abs(dv))   # sums of |terms|
    o, wsz, ob, _ = off[name]
    dw = g[o:o + wsz].reshape(dw_ref.shape)
    db = g[ob:ob + co]
    assert np.all(np.isfinite(dw)) and np.all(np.isfinite(db))
    err_w = np.abs(dw - dw_ref) - (1e-5 * dw_abs + 1e-30)
    err_b = np.abs(db - db_ref) - (1e-5 * db_abs + 1e-30)
    assert err_w.max() <= 0, (name, float(np.abs(dw - dw_ref).max()), float(dw_abs.max()))
    assert err_b.max() <= 0, (name, float(np.abs(db - db_ref).max()), float(db_abs.max()))
    # nothing outside the layer's slice was written
    rest = np.concatenate([g[:o], g[ob + co:]])
    assert np.all(np.isnan(rest))


DGRAD = [(i, name) for i, name in CONV3 if i != 0]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("layer,name", DGRAD)
def test_layer_dgrad(layer, name, masked, prec):
    """Data gradient: BF16 on the tensor cores with the flipped, transposed kernel (BF16 weights,
    FP32 accumulation, rounded to BF16 once), against the float64 oracle on the BF16 values,
    rounded once: within one BF16 ulp plus the FP32 summation bound over K = 9 C_out products,
    and almost all bit for bit.  F32: within 1e-5 of the largest value.  With a mask, outputs
    where the mask is not positive are exactly zero."""
    import torch
    from paper_2407_19097_gb300 import nrv
    flat = make_params(C0, seed=11 + layer)
    net = nrv.Net(C0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    _, _, ci, co = unet.layers(C0)[layer]
    n, h, w = 2, 7, 300
    rng = np.random.default_rng(200 + layer)
    dy = (rng.standard_normal((n, h, w, co)) * 0.1).astype(np.float32)
    mk = rng.standard_normal((n, h, w, ci)).astype(np.float32)
    mk[mk < 0] = 0.0                      # a ReLU output: zeros and positives
    dt = torch.bfloat16 if prec == 1 else torch.float32
    dyt = torch.from_numpy(dy).to(torch_dev()).to(dt).contiguous()
    mt = torch.from_numpy(mk).to(torch_dev()).to(dt).contiguous() if masked else None
    dx = torch.empty((n, h, w, ci), dtype=dt, device=torch_dev())
    net.layer_dgrad(layer, dyt, mt, n, h, w, prec, dx)
    torch.cuda.synchronize()
    got = dx.float().cpu().numpy().astype(np.float64)
    W, _ = unet.unflatten(flat.astype(np.float64), C0)[name]
    Wq = _bf16(W) if prec == 1 else W
    dv = _bf16(dy) if prec == 1 else dy.astype(np.float64)
    zero = np.zeros((n, h, w, ci))
    ref = unet.conv3_bwd(zero, Wq, dv)[0]
    S = unet.conv3_bwd(zero, np.abs(Wq), np.abs(dv))[0]
    if masked:
        keep = mk > 0
        ref = np.where(keep, ref, 0.0)
        assert np.all(got[~keep] == 0.0)
    if prec == 1:
        ref = _bf16(ref)
        K = 9 * co
        big = np.maximum(np.abs(got), np.abs(ref))
        ulp = np.exp2(np.floor(np.log2(np.maximum(big, 1e-30))) - 7)
        bound = ulp + K * 2.0 ** -24 / (1 - K * 2.0 ** -24) * S
        worst = float(np.max(np.abs(got - ref) / bound))
        exact = float(np.mean(got == ref))
        assert exact >= 0.99 and worst <= 1.0, (exact, worst)
    else:
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err <= 1e-5, err


UPCONV = [(i, name) for i, (name, kind, _, _) in enumerate(unet.layers(C0)) if kind == "convT2"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layer,name", UPCONV)
def test_upconv_wgrad(layer, name, prec):
    """Transposed conv weight and bias gradients (BF16: tensor cores with a parity view of the
    output gradient; F32: CUDA cores) against the oracle's convT2_bwd on the same values, within
    the FP32 summation bound.  Input 300 wide (three 128-pixel tiles, ragged) and enough rows
    that each K-split sums several tiles."""
    import torch
    from paper_2407_19097_gb300 import nrv
    net = nrv.Net(C0)
    net.set_params(torch.from_numpy(make_params(C0, seed=9)).to(torch_dev()))
    _, _, ci, co = unet.layers(C0)[layer]
    n, h, w = 2, 100, 300
    rng = np.random.default_rng(300 + layer)
    x = rng.standard_normal((n, h, w, ci)).astype(np.float32)
    dy = (rng.standard_normal((n, 2 * h, 2 * w, co)) * 0.1).astype(np.float32)
    dt = torch.bfloat16 if prec == 1 else torch.float32
    xt = torch.from_numpy(x).to(torch_dev()).to(dt).contiguous()
    dyt = torch.from_numpy(dy).to(torch_dev()).to(dt).contiguous()
    off, total = _offsets(C0)
    grad = torch.full((total,), float("nan"), device=torch_dev())
    net.layer_wgrad(layer, dyt, xt, None, n, h, w, prec, grad)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    xv = _bf16(x) if prec == 1 else x.astype(np.float64)
    dv = _bf16(dy) if prec == 1 else dy.astype(np.float64)
    wz = np.zeros(unet.weight_shape("convT2", ci, co))
    _, dw_ref, db_ref = unet.convT2_bwd(xv, wz, dv)
    _, dw_abs, db_abs = unet.convT2_bwd(np.abs(xv), wz, np.abs(dv))
    o, wsz, ob, _ = off[name]
    dw = g[o:o + wsz].reshape(dw_ref.shape)
    db = g[ob:ob + co]
    assert np.all(np.isfinite(dw)) and np.all(np.isfinite(db))
    assert np.all(np.abs(dw - dw_ref) <= 1e-5 * dw_abs + 1e-30), float(np.abs(dw - dw_ref).max())
    assert np.all(np.abs(db - db_ref) <= 1e-5 * db_abs + 1e-30), float(np.abs(db - db_ref).max())
    rest = np.concatenate([g[:o], g[ob + co:]])
    assert np.all(np.isnan(rest))



@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layer,name", UPCONV)
def test_upconv_dgrad(layer, name, prec):
    """Transposed conv data gradient, masked by the layer's input (a ReLU output): BF16 on the
    tensor cores (parity views of the output gradient, BF16 weights, FP32 accumulation, rounded
    once), against the float64 oracle on the BF16 values, rounded once: within one BF16 ulp plus
    the FP32 summation bound over K = 4 C_out products, and almost all bit for bit.  F32 (CUDA
    cores): within 1e-5 of the largest value.  Masked outputs are exactly zero."""
    import torch
    from paper_2407_19097_gb300 import nrv
    flat = make_params(C0, seed=13 + layer)
    net = nrv.Net(C0)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    _, _, ci, co = unet.layers(C0)[layer]
    n, h, w = 2, 5, 300
    rng = np.random.default_rng(400 + layer)
    dy = (rng.standard_normal((n, 2 * h, 2 * w, co)) * 0.1).astype(np.float32)
    mk = rng.standard_normal((n, h, w, ci)).astype(np.float32)
    mk[mk < 0] = 0.0
    dt = torch.bfloat16 if prec == 1 else torch.float32
    dyt = torch.from_numpy(dy).to(torch_dev()).to(dt).contiguous()
    mt = torch.from_numpy(mk).to(torch_dev()).to(dt).contiguous()
    dx = torch.empty((n, h, w, ci), dtype=dt, device=torch_dev())
    net.layer_dgrad(layer, dyt, mt, n, h, w, prec, dx)
    torch.cuda.synchronize()
    got = dx.float().cpu().numpy().astype(np.float64)
    W, _ = unet.unflatten(flat.astype(np.float64), C0)[name]
    Wq = _bf16(W) if prec == 1 else W
    dv = _bf16(dy) if prec == 1 else dy.astype(np.float64)
    zero = np.zeros((n, h, w, ci))
    ref = unet.convT2_bwd(zero, Wq, dv)[0]
    S = unet.convT2_bwd(zero, np.abs(Wq), np.abs(dv))[0]
    keep = mk > 0
    ref = np.where(keep, ref, 0.0)
    assert np.all(got[~keep] == 0.0)
    if prec == 1:
        ref = _bf16(ref)
        K = 4 * co
        big = np.maximum(np.abs(got), np.abs(ref))
        ulp = np.exp2(np.floor(np.log2(np.maximum(big, 1e-30))) - 7)
        bound = ulp + K * 2.0 ** -24 / (1 - K * 2.0 ** -24) * S
        worst = float(np.max(np.abs(got - ref) / bound))
        exact = float(np.mean(got == ref))
        assert exact >= 0.99 and worst <= 1.0, (exact, worst)
    else:
        err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
        assert err <= 1e-5, err
