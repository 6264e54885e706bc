"""Pins for the float64 U-Net oracle (Sec. 3.3): torch.nn.functional in float64 as a library
routine for forward and autograd backward, central finite differences, special cases, and
the parameter count worked out layer by layer."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import nrv_inputs as I
from oracle import unet


def _params(c0, seed=3):
    flat = []
    for t, (name, kind, ci, co) in enumerate(unet.layers(c0)):
        fi, fo = unet.fans(kind, ci, co)
        flat.append(I.xavier_uniform(seed, 1000 + t, unet.weight_shape(kind, ci, co), fi, fo).reshape(-1))
        # non-zero biases so that bias handling is exercised too
        flat.append((0.05 * I.normal_array(seed, 2000 + t, co)).astype(np.float32))
    return np.concatenate(flat).astype(np.float64)


def test_param_count_by_hand():
    # per 3x3 conv: 9*ci*co + co; per 2x2 transposed conv: 4*ci*co + co; head: 16*3 + 3
    conv = lambda ci, co: 9 * ci * co + co
    up = lambda ci, co: 4 * ci * co + co
    n = (conv(5, 16) + conv(16, 16) + conv(16, 32) + conv(32, 32) + conv(32, 64) + conv(64, 64)
         + conv(64, 128) + conv(128, 128) + up(128, 64) + conv(128, 64) + conv(64, 64)
         + up(64, 32) + conv(64, 32) + conv(32, 32) + up(32, 16) + conv(32, 16) + conv(16, 16)
         + 16 * 3 + 3)
    assert n == 482_355 == unet.param_count(5)


def _torch_unet(x_nhwc, flat, c0):
    """The same network written with torch.nn.functional (NCHW, float64)."""
    p = {}
    o = 0
    for name, kind, ci, co in unet.layers(c0):
        shp = unet.weight_shape(kind, ci, co)
        n = int(np.prod(shp))
        p[name] = (flat[o:o + n].view(shp), flat[o + n:o + n + co])
        o += n + co
    cr = lambda name, t: F.relu(F.conv2d(t, p[name][0], p[name][1], padding=1))
    x = x_nhwc.permute(0, 3, 1, 2)
    e0 = cr("e0b", cr("e0a", x))
    e1 = cr("e1b", cr("e1a", F.avg_pool2d(e0, 2)))
    e2 = cr("e2b", cr("e2a", F.avg_pool2d(e1, 2)))
    a = cr("e3b", cr("e3a", F.avg_pool2d(e2, 2)))
    for up, da, db, skip in (("up3", "d2a", "d2b", e2), ("up2", "d1a", "d1b", e1), ("up1", "d0a", "d0b", e0)):
        u = F.conv_transpose2d(a, p[up][0], p[up][1], stride=2)
        a = cr(db, cr(da, torch.cat([u, skip], 1)))
    w, b = p["head"]
    y = F.conv2d(a, w[:, :, None, None], b)
    return y.permute(0, 2, 3, 1)


@pytest.mark.parametrize("c0,h,w", [(5, 16, 24), (7, 8, 16)])
def test_forward_and_backward_match_torch_float64(c0, h, w):
    rng = np.random.default_rng(c0)
    x = rng.standard_normal((2, h, w, c0))
    flat = _params(c0)
    y, s = unet.forward(x, unet.unflatten(flat, c0), save=True)
    xt = torch.tensor(x, requires_grad=True)
    ft = torch.tensor(flat, requires_grad=True)
    yt = _torch_unet(xt, ft, c0)
    np.testing.assert_allclose(y, yt.detach().numpy(), rtol=1e-12, atol=1e-12)
    dy = rng.standard_normal(y.shape)
    (yt * torch.tensor(dy)).sum().backward()
    g, dx = unet.backward(dy, unet.unflatten(flat, c0), s)
    np.testing.assert_allclose(unet.flatten(g, c0), ft.grad.numpy(), rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-10, atol=1e-11)


def test_finite_differences():
    c0 = 5
    rng = np.random.default_rng(11)
    x = rng.standard_normal((1, 8, 16, c0))
    flat = _params(c0, seed=9)
    dy = rng.standard_normal((1, 8, 16, 3))
    loss = lambda f, xx: float((unet.forward(xx, unet.unflatten(f, c0)) * dy).sum())
    y, s = unet.forward(x, unet.unflatten(flat, c0), save=True)
    g, dx = unet.backward(dy, unet.unflatten(flat, c0), s)
    gf = unet.flatten(g, c0)
    h = 1e-6
    idx = rng.choice(flat.size, 60, replace=False)
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        fd = (loss(fp, x) - loss(fm, x)) / (2 * h)
        assert abs(fd - gf[i]) <= 1e-6 * max(1.0, abs(gf[i])), (i, fd, gf[i])
    for _ in range(10):
        j = tuple(int(rng.integers(n)) for n in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (loss(flat, xp) - loss(flat, xm)) / (2 * h)
        assert abs(fd - dx[j]) <= 1e-6 * max(1.0, abs(dx[j]))


def test_identity_tap_and_one_by_one_head():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 5, 7, 4))
    w = np.zeros((4, 4, 3, 3))
    w[:, :, 1, 1] = np.eye(4)
    np.testing.assert_array_equal(unet.conv3(x, w, np.zeros(4)), x)
    # a shift tap moves the image by one pixel with zero fill
    w2 = np.zeros((4, 4, 3, 3))
    w2[:, :, 1, 2] = np.eye(4)
    y = unet.conv3(x, w2, np.zeros(4))
    np.testing.assert_array_equal(y[:, :, :-1], x[:, :, 1:])
    assert np.all(y[:, :, -1] == 0)
    wh = rng.standard_normal((3, 4))
    np.testing.assert_allclose(unet.conv1(x, wh, np.zeros(3)), np.einsum("nhwc,oc->nhwo", x, wh))
    # pooling of a constant is the constant; transposed conv of a delta is the kernel
    np.testing.assert_array_equal(unet.avgpool2(np.full((1, 4, 4, 2), 3.0)), np.full((1, 2, 2, 2), 3.0))
    d = np.zeros((1, 2, 2, 1))
    d[0, 1, 0, 0] = 1.0
    wt = rng.standard_normal((1, 2, 2, 2))
    yt = unet.convT2(d, wt, np.zeros(2))
    np.testing.assert_array_equal(yt[0, 2:4, 0:2, :], wt[0].transpose(1, 2, 0))


def test_l1_loss_and_adam_match_torch():
    y = np.array([1.0, 2.0, 3.0, 4.0])
    t = np.array([1.5, 2.0, 2.0, 5.0])
    l, g = unet.l1_loss(y, t)
    assert l == (0.5 + 0 + 1 + 1) / 4
    np.testing.assert_array_equal(g, [-0.25, 0.0, 0.25, -0.25])
    rng = np.random.default_rng(0)
    p0 = rng.standard_normal(50)
    pt = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 6):
        grad = rng.standard_normal(50)
        pt.grad = torch.tensor(grad)
        opt.step()
        p, m, v = unet.adam_step(p, grad, m, v, step)
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=0, atol=1e-15)


class _RoundBoth(torch.autograd.Function):
    """Rounds a float64 tensor to bfloat16 values in forward and its gradient in backward."""

    @staticmethod
    def forward(ctx, t):
        return t.to(torch.bfloat16).to(torch.float64)

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(torch.float64)


def _torch_unet_rounded(x_nhwc, flat, c0):
    """torch.nn.functional U-Net with every stored tensor (and its gradient) rounded to bf16."""
    R = _RoundBoth.apply
    p, o = {}, 0
    for name, kind, ci, co in unet.layers(c0):
        shp = unet.weight_shape(kind, ci, co)
        n = int(np.prod(shp))
        p[name] = (flat[o:o + n].view(shp), flat[o + n:o + n + co])
        o += n + co
    cr = lambda name, t: R(F.relu(F.conv2d(t, p[name][0], p[name][1], padding=1)))
    x = R(x_nhwc).permute(0, 3, 1, 2)
    e0 = cr("e0b", cr("e0a", x))
    e1 = cr("e1b", cr("e1a", R(F.avg_pool2d(e0, 2))))
    e2 = cr("e2b", cr("e2a", R(F.avg_pool2d(e1, 2))))
    a = cr("e3b", cr("e3a", R(F.avg_pool2d(e2, 2))))
    for up, da, db, skip in (("up3", "d2a", "d2b", e2), ("up2", "d1a", "d1b", e1), ("up1", "d0a", "d0b", e0)):
        u = R(F.conv_transpose2d(a, p[up][0], p[up][1], stride=2))
        a = cr(db, cr(da, R(torch.cat([u, skip], 1))))
    w, b = p["head"]
    return F.conv2d(a, w[:, :, None, None], b).permute(0, 2, 3, 1)


def test_storage_rounding_hook_matches_torch():
    """forward/backward with q = bf16 rounding equal torch float64 with bf16 rounding of every
    stored tensor and of every gradient passed between layers."""
    import oracle
    c0 = 5
    q = lambda t: oracle.bf16_value(oracle.bf16_bits(np.asarray(t, np.float32))).astype(np.float64)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((2, 16, 24, c0))
    flat = _params(c0, seed=13)
    y, s = unet.forward(x, unet.unflatten(flat, c0), save=True, q=q)
    xt = torch.tensor(x, requires_grad=True)
    ft = torch.tensor(flat, requires_grad=True)
    yt = _torch_unet_rounded(xt, ft, c0)
    np.testing.assert_allclose(y, yt.detach().numpy(), rtol=1e-9, atol=1e-12)
    dy = rng.standard_normal(y.shape) * 1e-2
    (yt * torch.tensor(dy)).sum().backward()
    g, dx = unet.backward(dy, unet.unflatten(flat, c0), s, q=q)
    np.testing.assert_allclose(unet.flatten(g, c0), ft.grad.numpy(), rtol=1e-8, atol=1e-12)
    # with q = identity the hook changes nothing
    y2 = unet.forward(x, unet.unflatten(flat, c0), q=lambda t: t)
    np.testing.assert_array_equal(y2, unet.forward(x, unet.unflatten(flat, c0)))
    assert 0.0 < unet.relu_margin(s) < 1.0


def test_recon_tv_loss_closed_forms():
    """Eq. (1) without its perceptual term: a horizontal ramp y = a x has total variation a
    (all horizontal differences a, no vertical ones); a constant offset c gives L2 = c^2 and
    L1 = |c|."""
    n, h, w = 2, 5, 7
    a = 0.25
    y = np.broadcast_to((a * np.arange(w))[None, None, :, None], (n, h, w, 3)).copy()
    loss, _ = unet.recon_tv_loss(y, y, tv=1.0)
    assert abs(loss - a) < 1e-15
    c = -0.3
    loss, g = unet.recon_tv_loss(y + c, y, l1=1.0, l2=1.0)
    assert abs(loss - (abs(c) + c * c)) < 1e-15
    np.testing.assert_allclose(g, (np.sign(c) + 2 * c) / y.size, rtol=1e-15)


def test_recon_tv_loss_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    y = rng.standard_normal((2, 4, 5, 3))
    t = rng.standard_normal((2, 4, 5, 3))
    wts = dict(l1=0.7, l2=1.3, tv=0.4)
    _, g = unet.recon_tv_loss(y, t, **wts)
    h = 1e-7
    for idx in [(0, 0, 0, 0), (1, 3, 4, 2), (0, 2, 1, 1), (1, 0, 4, 0), (0, 3, 2, 2)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += h
        ym[idx] -= h
        fd = (unet.recon_tv_loss(yp, t, **wts)[0] - unet.recon_tv_loss(ym, t, **wts)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])
