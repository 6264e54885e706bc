"""The learned part end to end (Sec. 3.3 training; Tab. 1's comparison of the rasterizer alone
against the full method): the U-Net is trained on the GPU by the library's own BF16 forward and
backward kernels (nrv_train_step: L1 loss, Adam lr 1e-3) on pairs of G-buffers, rendered by the
library's rasterizer, and targets from the CPU Gaussian-splat renderer that stands in for the
paper's Gaussian Renderer.  On held-out views the trained network must beat the method without
it -- each pixel coloured by the transfer function of its winning point, black where empty --
in PSNR against the splatted targets."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import make_params, torch_dev, upload_scene
from oracle import metrics

pytestmark = pytest.mark.gpu


def test_training_beats_the_rasterizer_alone():
    import torch
    from paper_2407_19097_gb300 import nrv
    dev = torch_dev()
    sc = I.trajectory_scene(3000, 350, seed=2)              # 1.05M trajectory points
    colours = I.point_colours(sc)
    size, n_views, n_train = 96, 24, 20
    views = I.hemisphere_views(sc, n_views, size, size, seed=5)
    scene = upload_scene(sc)
    c0 = len(sc.channels) + 2
    # one pack normalisation for every view: the scene's depth range seen from the first one
    ds, do = I.depth_normalisation(sc, views[0])
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    netins, targets, baselines = [], [], []
    for v in views:
        key = torch.empty((size, size), dtype=torch.int64, device=dev)
        depth = torch.empty((size, size), dtype=torch.int32, device=dev)
        mask = torch.empty((size, size), dtype=torch.uint8, device=dev)
        gattr = torch.empty((sc.n_words, size, size), dtype=torch.int32, device=dev)
        nrv.rasterize(scene, [v], [key], [depth], [mask], [gattr])
        x = torch.empty((size, size, 8), dtype=torch.bfloat16, device=dev)
        nrv.pack(depth, mask, gattr, size, size, desc, nrv.PREC_BF16, x)
        netins.append(x)
        targets.append(np.clip(oracle.splat(sc.xyz, v, colours), 0.0, 1.0).astype(np.float32))
        # the method without the network: transfer-function colour of the winning point
        k = key.cpu().numpy().view(np.uint64)
        hit = k != np.uint64(0xFFFFFFFFFFFFFFFF)
        base = np.zeros((size, size, 3), np.float32)
        base[hit] = colours[(k[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)]
        baselines.append(base)
    X = torch.stack(netins)                                  # [V, H, W, 8] BF16
    T = torch.from_numpy(np.stack(targets)).to(dev)          # [V, H, W, 3]
    net = nrv.Net(c0)
    p = torch.from_numpy(make_params(c0, seed=1)).to(dev)
    net.set_params(p)
    g, m, v = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    loss = torch.zeros(1, device=dev)
    batch = 8
    losses = []
    for step in range(1, 401):
        idx = torch.tensor([int(I.uniform(3, 600, step * batch + b) * n_train) for b in range(batch)],
                           device=dev)
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        net.train_step(p, g, m, v, step, 1e-3, xb, tb, batch, size, size, nrv.PREC_BF16, loss)
        if step % 50 == 0:
            losses.append(loss.item())
    assert losses[-1] < losses[0]
    # held-out views
    out = torch.empty((n_views - n_train, size, size, 3), device=dev)
    net.shade(X[n_train:].contiguous(), n_views - n_train, size, size, nrv.PREC_BF16, out)
    torch.cuda.synchronize()
    y = np.clip(out.cpu().numpy(), 0.0, 1.0)
    p_net = np.mean([metrics.psnr(y[i], targets[n_train + i]) for i in range(n_views - n_train)])
    p_base = np.mean([metrics.psnr(baselines[n_train + i], targets[n_train + i])
                      for i in range(n_views - n_train)])
    s_net = np.mean([metrics.ssim(y[i], targets[n_train + i]) for i in range(n_views - n_train)])
    s_base = np.mean([metrics.ssim(baselines[n_train + i], targets[n_train + i])
                      for i in range(n_views - n_train)])
    print(f"held-out PSNR: network {p_net:.2f} dB vs rasterizer alone {p_base:.2f} dB; "
          f"SSIM {s_net:.3f} vs {s_base:.3f}; loss {losses}")
    assert p_net > p_base + 1.0
