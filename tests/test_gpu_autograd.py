"""The network behind torch.autograd (Sec. 3.3 training): NrvUNet's gradient against the float64
oracle, a loop through NrvUNet + nrv_l1 + NrvAdam bit-identical to nrv_train_step step by step,
and torch.optim.Adam driving the same module."""
import numpy as np
import pytest

from gpu_util import torch_dev
from oracle import unet
from test_gpu_net import _clean_case, _input

pytestmark = pytest.mark.gpu


def test_autograd_gradient_matches_oracle_fp32():
    import torch
    from paper_2407_19097_gb300 import nrv
    from paper_2407_19097_gb300.autograd import NrvUNet
    c0, n, h, w = 5, 2, 16, 24
    flat, x, s, q = _clean_case(nrv.PREC_F32, c0, n, h, w)
    dev = torch_dev()
    mod = NrvUNet(c0, nrv.PREC_F32)
    with torch.no_grad():
        mod.params.copy_(torch.from_numpy(flat))
    rgb = mod(torch.from_numpy(x).to(dev), h, w)
    dy = (np.random.default_rng(4).standard_normal((n, h, w, 3)) * 1e-2).astype(np.float32)
    rgb.backward(torch.from_numpy(dy).to(dev))
    gr, _ = unet.backward(dy.astype(np.float64), unet.unflatten(flat, c0), s)
    got = mod.params.grad.cpu().numpy().astype(np.float64)
    o = 0
    for name, kind, ci, co in unet.layers(c0):
        for ref in gr[name]:
            g = got[o:o + ref.size]
            err = np.linalg.norm(g - ref.ravel()) / max(np.linalg.norm(ref), 1e-30)
            assert err <= 1e-4, (name, err)
            o += ref.size
    assert o == got.size
    y, _ = unet.forward(x[..., :c0].astype(np.float64), unet.unflatten(flat, c0), save=True)
    assert np.abs(rgb.detach().cpu().numpy() - y).max() <= 1e-4


@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_loop_equals_train_step(prec):
    """forward -> nrv_l1 -> backward -> NrvAdam through torch.autograd runs the same kernels on
    the same data as nrv_train_step: parameters and losses bit-identical after every step."""
    import torch
    from paper_2407_19097_gb300 import nrv
    from paper_2407_19097_gb300.autograd import NrvAdam, NrvUNet, nrv_l1
    c0, n, h, w = 5, 2, 32, 40
    dev = torch_dev()
    x = torch.from_numpy(_input(n, h, w, c0, seed=8)).to(dev)
    if prec == nrv.PREC_BF16:
        x = x.to(torch.bfloat16)
    tgt = torch.from_numpy(np.random.default_rng(9).uniform(0, 1, (n, h, w, 3)).astype(np.float32)).to(dev)
    mod = NrvUNet(c0, prec, seed=3)
    opt = NrvAdam(mod.parameters(), lr=1e-3)
    ref_net = nrv.Net(c0)
    p = torch.empty_like(mod.params.detach())
    ref_net.init_params(3, p)
    assert torch.equal(p, mod.params.detach())
    g, m, v = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    loss_ref = torch.zeros(1, device=dev)
    for step in range(1, 5):
        ref_net.train_step(p, g, m, v, step, 1e-3, x, tgt, n, h, w, prec, loss_ref)
        opt.zero_grad()
        loss = nrv_l1(mod(x, h, w), tgt)
        loss.backward()
        opt.step()
        torch.cuda.synchronize()
        assert loss.item() == loss_ref.item(), step
        assert torch.equal(mod.params.detach(), p), step
        assert torch.equal(mod.params.grad, g), step


def test_torch_adam_through_module():
    """torch.optim.Adam on NrvUNet (FP32): the trajectory agrees with NrvAdam's to rounding and
    the loss falls."""
    import torch
    from paper_2407_19097_gb300 import nrv
    from paper_2407_19097_gb300.autograd import NrvAdam, NrvUNet, nrv_l1
    c0, n, h, w = 5, 2, 32, 32
    dev = torch_dev()
    x = torch.from_numpy(_input(n, h, w, c0, seed=10)).to(dev)
    tgt = torch.from_numpy(np.random.default_rng(11).uniform(0, 1, (n, h, w, 3)).astype(np.float32)).to(dev)
    a, b = NrvUNet(c0, nrv.PREC_F32, seed=4), NrvUNet(c0, nrv.PREC_F32, seed=4)
    oa, ob = torch.optim.Adam(a.parameters(), lr=1e-3), NrvAdam(b.parameters(), lr=1e-3)
    first = last = None
    for step in range(30):
        for mod, opt in ((a, oa), (b, ob)):
            opt.zero_grad()
            loss = nrv_l1(mod(x, h, w), tgt)
            loss.backward()
            opt.step()
            if mod is a:
                first = loss.item() if first is None else first
                last = loss.item()
        torch.cuda.synchronize()
        if step < 3:
            np.testing.assert_allclose(a.params.detach().cpu().numpy(), b.params.detach().cpu().numpy(),
                                       rtol=0, atol=1e-6)
    assert last < first


def test_backward_after_second_forward_raises():
    import torch
    from paper_2407_19097_gb300 import nrv
    from paper_2407_19097_gb300.autograd import NrvUNet
    c0, n, h, w = 5, 1, 16, 16
    x = torch.from_numpy(_input(n, h, w, c0, seed=1)).to(torch_dev())
    mod = NrvUNet(c0, nrv.PREC_F32)
    y1 = mod(x, h, w)
    mod(x, h, w)
    with pytest.raises(RuntimeError, match="another forward"):
        y1.sum().backward()
