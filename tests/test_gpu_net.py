"""GPU parity of the post-processing U-Net (Sec. 3.3) against the float64 oracle: FP32 forward
within 1e-4, BF16 forward at PSNR >= 45 dB and max abs <= 2e-2, gradients of the backward pass
per tensor, L1 loss and Adam."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import make_params, psnr_range, torch_dev
from oracle import unet

pytestmark = pytest.mark.gpu


def _input(n, h, w, c0, seed=0):
    """Packed-looking network input: covered pixels with z-scored channels, depth, mask."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n, h, w, 8), np.float32)
    cov = rng.uniform(0, 1, (n, h, w)) < 0.6
    x[..., :c0 - 2] = rng.standard_normal((n, h, w, c0 - 2)).astype(np.float32)
    x[..., c0 - 2] = rng.uniform(0, 1, (n, h, w)).astype(np.float32)
    x[..., c0 - 1] = 1.0
    x[~cov] = 0.0
    return x


def _net(c0, flat):
    import torch
    from paper_2407_19097_gb300 import nrv
    net = nrv.Net(c0)
    p = torch.from_numpy(flat).to(torch_dev())
    net.set_params(p)
    return net, p


@pytest.mark.parametrize("c0,n,h,w", [(5, 2, 64, 96), (7, 1, 40, 136), (6, 1, 120, 40)])
def test_forward_fp32(c0, n, h, w):
    import torch
    from paper_2407_19097_gb300 import nrv
    flat = make_params(c0, seed=c0, bias_sigma=0.05)
    net, _ = _net(c0, flat)
    hn, wn = nrv.lib().nrv_pad8(h), nrv.lib().nrv_pad8(w)
    x = _input(n, hn, wn, c0, seed=1)
    xt = torch.from_numpy(x).to(torch_dev())
    rgb = torch.empty((n, h, w, 3), device=torch_dev())
    net.shade(xt, n, h, w, nrv.PREC_F32, rgb)
    ref = unet.forward(x[..., :c0].astype(np.float64), unet.unflatten(flat, c0))[:, :h, :w]
    torch.cuda.synchronize()
    err = np.abs(rgb.cpu().numpy() - ref).max()
    assert err <= 1e-4, err


@pytest.mark.parametrize("c0,n,h,w", [(5, 2, 64, 96), (7, 1, 136, 264)])
def test_forward_bf16(c0, n, h, w):
    import torch
    from paper_2407_19097_gb300 import nrv
    flat = make_params(c0, seed=c0 + 10, bias_sigma=0.05)
    net, _ = _net(c0, flat)
    hn, wn = nrv.lib().nrv_pad8(h), nrv.lib().nrv_pad8(w)
    x = _input(n, hn, wn, c0, seed=2)
    xb = torch.from_numpy(x).to(torch_dev()).to(torch.bfloat16)
    xin = xb.float().cpu().numpy()          # the oracle sees exactly the BF16 input values
    rgb = torch.empty((n, h, w, 3), device=torch_dev())
    net.shade(xb, n, h, w, nrv.PREC_BF16, rgb)
    ref = unet.forward(xin[..., :c0].astype(np.float64), unet.unflatten(flat, c0))[:, :h, :w]
    torch.cuda.synchronize()
    got = rgb.cpu().numpy()
    err = np.abs(got - ref).max()
    p = psnr_range(got, ref)
    assert err <= 2e-2 and p >= 45.0, (err, p)
    # every 3x3 and transposed convolution ran on the tensor cores
    kinds = [k for (_, k, _, _, _, _) in nrv.layer_table(c0)]
    assert [b for b, k in zip(net.backends(), kinds) if k in (0, 1)] == [1] * 17, net.backends()


def _bf16(t):
    return oracle.bf16_value(oracle.bf16_bits(np.asarray(t, np.float32))).astype(np.float64)


def _fwd_params(flat, c0, prec):
    """Weights as each forward kernel uses them: the BF16 path's 3x3 convolutions read BF16
    weights; transposed convs, the head and every backward kernel read the FP32 master copy."""
    P = unet.unflatten(flat, c0)
    if prec == 1:
        P = {k: ((_bf16(w), b) if w.shape[2:] == (3, 3) else (w, b)) for k, (w, b) in P.items()}
    return P


def _clean_case(prec, c0=5, n=2, h=16, w=24, margin=1e-6):
    """First seeded (weights, input) whose ReLU decisions all clear zero by `margin` (relative),
    so that FP32/FP64 accumulation order cannot flip one; the oracle decides."""
    q = _bf16 if prec == 1 else None
    for sd in range(64):
        flat = make_params(c0, seed=100 + sd, bias_sigma=0.05)
        x = _input(n, h, w, c0, seed=sd)
        xin = _bf16(x) if prec == 1 else x.astype(np.float64)
        y, s = unet.forward(xin[..., :c0], _fwd_params(flat, c0, prec), save=True, q=q)
        if unet.relu_margin(s) >= margin:
            return flat, x, s, q
    raise AssertionError("no seed with clear ReLU decisions")


def _grad_case(prec, tol):
    import torch
    from paper_2407_19097_gb300 import nrv
    c0, n, h, w = 5, 2, 16, 24
    flat, x, s, q = _clean_case(prec, c0, n, h, w)
    net, p = _net(c0, flat)
    dev = torch_dev()
    xt = torch.from_numpy(x).to(dev)
    if prec == nrv.PREC_BF16:
        xt = xt.to(torch.bfloat16)
    rgb = torch.empty((n, h, w, 3), device=dev)
    net.forward_train(xt, n, h, w, prec, rgb)
    rng = np.random.default_rng(4)
    dy = (rng.standard_normal((n, h, w, 3)) * 1e-2).astype(np.float32)
    g = torch.zeros_like(p)
    net.backward(torch.from_numpy(dy).to(dev), g)
    gr, _ = unet.backward(dy.astype(np.float64), unet.unflatten(flat, c0), s, q=q)
    torch.cuda.synchronize()
    gg = g.cpu().numpy().astype(np.float64)
    o = 0
    errs = {}
    for name, kind, ci, co in unet.layers(c0):
        wref, bref = gr[name]
        for part, ref in (("w", wref), ("b", bref)):
            got = gg[o:o + ref.size]
            errs[name + "." + part] = np.linalg.norm(got - ref.ravel()) / max(np.linalg.norm(ref), 1e-30)
            o += ref.size
    assert o == gg.size
    report = " ".join(f"{k}={v:.2e}" for k, v in errs.items())
    assert all(v <= tol for v in errs.values()), report
    ref_all = unet.flatten(gr, c0)
    cos = float(gg @ ref_all / (np.linalg.norm(gg) * np.linalg.norm(ref_all)))
    assert cos >= 0.999 if prec == nrv.PREC_F32 else cos >= 0.99, cos


def test_backward_fp32():
    """FP32 backward vs the float64 oracle."""
    from paper_2407_19097_gb300 import nrv
    _grad_case(nrv.PREC_F32, 1e-4)


def test_backward_bf16():
    """BF16 backward vs the oracle at BF16 storage precision: the same tensors rounded to BF16
    where the kernels store them, FP32/FP64 accumulation inside each layer.  Across 18 layers
    the two accumulation orders round a few stored values differently and those flip ReLU
    decisions downstream, so the bound is statistical: <= 0.15 relative per tensor and a
    cosine >= 0.99 for the whole gradient.  Every layer's weight and data gradients are
    checked tightly one layer at a time in test_gpu_layer_grad.py."""
    from paper_2407_19097_gb300 import nrv
    _grad_case(nrv.PREC_BF16, 0.15)


def test_backward_bf16_training_shape():
    """The BF16 backward at the training configuration's shape (16 crops of 256 x 256, Sec. 3.3
    training) against the oracle at BF16 storage precision, seeded weights and inputs: the same
    statistical bound as the small case (<= 0.15 relative per tensor, cosine >= 0.99)."""
    import torch
    from paper_2407_19097_gb300 import nrv
    c0, n, h, w = 5, 16, 256, 256
    flat = make_params(c0, seed=7, bias_sigma=0.05)
    x = _input(n, h, w, c0, seed=11)
    q = _bf16
    _, s = unet.forward(_bf16(x)[..., :c0], _fwd_params(flat, c0, 1), save=True, q=q)
    net, p = _net(c0, flat)
    dev = torch_dev()
    xt = torch.from_numpy(x).to(dev).to(torch.bfloat16)
    rgb = torch.empty((n, h, w, 3), device=dev)
    net.forward_train(xt, n, h, w, nrv.PREC_BF16, rgb)
    rng = np.random.default_rng(4)
    dy = (rng.standard_normal((n, h, w, 3)) * 1e-2).astype(np.float32)
    g = torch.zeros_like(p)
    net.backward(torch.from_numpy(dy).to(dev), g)
    gr, _ = unet.backward(dy.astype(np.float64), unet.unflatten(flat, c0), s, q=q)
    torch.cuda.synchronize()
    gg = g.cpu().numpy().astype(np.float64)
    o = 0
    errs = {}
    for name, kind, ci, co in unet.layers(c0):
        wref, bref = gr[name]
        for part, ref in (("w", wref), ("b", bref)):
            got = gg[o:o + ref.size]
            errs[name + "." + part] = np.linalg.norm(got - ref.ravel()) / max(np.linalg.norm(ref), 1e-30)
            o += ref.size
    assert o == gg.size
    report = " ".join(f"{k}={v:.2e}" for k, v in errs.items())
    print(report)
    assert all(v <= 0.15 for v in errs.values()), report
    ref_all = unet.flatten(gr, c0)
    cos = float(gg @ ref_all / (np.linalg.norm(gg) * np.linalg.norm(ref_all)))
    assert cos >= 0.99, cos


def test_l1_and_adam():
    import torch
    from paper_2407_19097_gb300 import nrv
    dev = torch_dev()
    rng = np.random.default_rng(5)
    y = rng.standard_normal(100_003).astype(np.float32)
    t = y.copy()
    t[::3] += rng.standard_normal(t[::3].shape).astype(np.float32)
    yt, tt = torch.from_numpy(y).to(dev), torch.from_numpy(t).to(dev)
    loss = torch.zeros(1, device=dev)
    dy = torch.empty_like(yt)
    nrv.l1_loss(yt, tt, loss, dy)
    lref, gref = unet.l1_loss(y, t)
    torch.cuda.synchronize()
    assert abs(loss.item() - lref) <= 1e-6 * max(1.0, lref)
    np.testing.assert_allclose(dy.cpu().numpy(), gref, rtol=1e-6, atol=0)
    p0 = rng.standard_normal(5000).astype(np.float32)
    pt = torch.from_numpy(p0).to(dev)
    m = torch.zeros_like(pt)
    v = torch.zeros_like(pt)
    pr, mr, vr = p0.astype(np.float64), np.zeros(5000), np.zeros(5000)
    for step in range(1, 4):
        gnp = rng.standard_normal(5000).astype(np.float32)
        nrv.adam_step(pt, torch.from_numpy(gnp).to(dev), m, v, step)
        pr, mr, vr = unet.adam_step(pr, gnp.astype(np.float64), mr, vr, step)
    torch.cuda.synchronize()
    np.testing.assert_allclose(pt.cpu().numpy(), pr, rtol=0, atol=1e-6)


def test_training_reduces_loss():
    import torch
    from paper_2407_19097_gb300 import nrv
    c0, n, h, w = 5, 4, 32, 32
    flat = make_params(c0, seed=3)
    net, p = _net(c0, flat)
    dev = torch_dev()
    x = torch.from_numpy(_input(n, h, w, c0, seed=6)).to(dev).to(torch.bfloat16)
    tgt = torch.from_numpy(np.random.default_rng(7).uniform(0, 1, (n, h, w, 3)).astype(np.float32)).to(dev)
    g, m, v = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    loss = torch.zeros(1, device=dev)
    losses = []
    for step in range(1, 61):
        net.train_step(p, g, m, v, step, 1e-3, x, tgt, n, h, w, nrv.PREC_BF16, loss)
        losses.append(loss.item())
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
