"""The reconstruction + total-variation loss (Eq. 1 without its perceptual term) against the
float64 oracle, its L1 special case against nrv_l1_loss, and training with it."""
import numpy as np
import pytest

from gpu_util import make_params, torch_dev
from oracle import unet

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,wts", [((2, 37, 53, 3), (0.7, 1.3, 0.4)), ((1, 1, 9, 3), (0.0, 1.0, 2.0)),
                                       ((3, 16, 1, 3), (0.5, 0.0, 1.0))])
def test_recon_loss_vs_oracle(shape, wts):
    import torch
    from paper_2407_19097_gb300 import nrv
    rng = np.random.default_rng(5)
    y = rng.standard_normal(shape).astype(np.float32)
    t = rng.standard_normal(shape).astype(np.float32)
    t.reshape(-1)[::11] = y.reshape(-1)[::11]                # exact zeros of y - t
    yt, tt = torch.from_numpy(y).to(torch_dev()), torch.from_numpy(t).to(torch_dev())
    loss, dy = torch.zeros(1, device=torch_dev()), torch.empty_like(yt)
    nrv.recon_loss(yt, tt, wts, loss, dy)
    lref, gref = unet.recon_tv_loss(y, t, *wts)
    torch.cuda.synchronize()
    assert abs(loss.item() - lref) <= 1e-5 * max(1.0, abs(lref)), (loss.item(), lref)
    np.testing.assert_allclose(dy.cpu().numpy(), gref, rtol=1e-5, atol=1e-6 / y.size)


def test_recon_loss_l1_case_equals_l1_loss():
    import torch
    from paper_2407_19097_gb300 import nrv
    rng = np.random.default_rng(6)
    y = torch.from_numpy(rng.standard_normal((2, 30, 40, 3)).astype(np.float32)).to(torch_dev())
    t = torch.from_numpy(rng.standard_normal((2, 30, 40, 3)).astype(np.float32)).to(torch_dev())
    la, lb = torch.zeros(1, device=torch_dev()), torch.zeros(1, device=torch_dev())
    da, db = torch.empty_like(y), torch.empty_like(y)
    nrv.recon_loss(y, t, (1.0, 0.0, 0.0), la, da)
    nrv.l1_loss(y, t, lb, db)
    torch.cuda.synchronize()
    assert torch.equal(da, db)
    assert abs(la.item() - lb.item()) <= 1e-6 * lb.item()


def test_training_with_l2_tv_loss():
    import torch
    from paper_2407_19097_gb300 import nrv
    from test_gpu_net import _input
    c0, n, h, w = 5, 4, 32, 32
    net = nrv.Net(c0)
    p = torch.from_numpy(make_params(c0, seed=3)).to(torch_dev())
    net.set_params(p)
    net.set_loss((0.0, 1.0, 0.01))
    x = torch.from_numpy(_input(n, h, w, c0, seed=6)).to(torch_dev()).to(torch.bfloat16)
    tgt = torch.from_numpy(np.random.default_rng(7).uniform(0, 1, (n, h, w, 3)).astype(np.float32)).to(torch_dev())
    g, m, v = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    loss = torch.zeros(1, device=torch_dev())
    losses = []
    for step in range(1, 61):
        net.train_step(p, g, m, v, step, 1e-3, x, tgt, n, h, w, nrv.PREC_BF16, loss)
        losses.append(loss.item())
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
    with pytest.raises(nrv.NrvError):
        net.set_loss((1.0, -1.0, 0.0))
