"""Whole frames through nrv_render_batch: several views of uneven size in one call, first run
eagerly and captured, later calls replayed from the CUDA graph with moved cameras.  Every frame
must equal, bit for bit, the same views rendered step by step through nrv_rasterize, nrv_pack
and nrv_shade; and the image must match the float64 oracle pipeline (render, resolve, pack,
U-Net) at PSNR >= 45 dB."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import make_params, psnr_range, torch_dev, upload_scene
from oracle import unet

pytestmark = pytest.mark.gpu


def _step_by_step(scene, net, sc, view, prec):
    import torch
    from paper_2407_19097_gb300 import nrv
    dev = torch_dev()
    H, W = view.height, view.width
    keys = [torch.empty((H, W), dtype=torch.int64, device=dev)]
    depth = [torch.empty((H, W), dtype=torch.int32, device=dev)]
    mask = [torch.empty((H, W), dtype=torch.uint8, device=dev)]
    gattr = [torch.empty((sc.n_words, H, W), dtype=torch.int32, device=dev)]
    nrv.rasterize(scene, [view], keys, depth, mask, gattr)
    ds, do = I.depth_normalisation(sc, view)
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    hn, wn = nrv.lib().nrv_pad8(H), nrv.lib().nrv_pad8(W)
    dt = torch.bfloat16 if prec == nrv.PREC_BF16 else torch.float32
    netin = torch.empty((hn, wn, 8), dtype=dt, device=dev)
    nrv.pack(depth[0], mask[0], gattr[0], H, W, desc, prec, netin)
    rgb = torch.empty((H, W, 3), device=dev)
    net.shade(netin, 1, H, W, prec, rgb)
    return rgb


@pytest.mark.parametrize("prec", [0, 1])
def test_render_batch_replay_matches_step_by_step(prec):
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.terrain_scene(600, seed=7)
    c0 = len(sc.channels) + 2
    scene = upload_scene(sc)
    net = nrv.Net(c0)
    flat = make_params(c0, seed=4, bias_sigma=0.05)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    sizes = [(216, 216), (192, 108), (96, 54)]
    outs = [torch.empty((h, w, 3), device=torch_dev()) for (w, h) in sizes]
    for frame, seed in enumerate((11, 11, 23, 37)):
        views = I.orbit_views(sc, sizes, seed=seed)
        # one pack descriptor for the batch: depth range of the first view
        ds, do = I.depth_normalisation(sc, views[0])
        desc = nrv.make_pack_desc(sc.channels, ds, do)
        nrv.render_batch(scene, net, desc, views, outs, prec)
        torch.cuda.synchronize()
        for v, o in zip(views, outs):
            # the step-by-step path packs with each view's own depth range; use the batch's
            ref = _step_by_step_with(scene, net, sc, v, prec, ds, do)
            assert torch.equal(o, ref), f"frame {frame}: batch differs from step-by-step"
    nrv.sync_status()


def _step_by_step_with(scene, net, sc, view, prec, ds, do):
    orig = I.depth_normalisation
    try:
        I.depth_normalisation = lambda s, v: (ds, do)
        return _step_by_step(scene, net, sc, view, prec)
    finally:
        I.depth_normalisation = orig


def test_render_batch_matches_oracle_pipeline():
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.trajectory_scene(2000, 35, seed=2)
    c0 = len(sc.channels) + 2
    scene = upload_scene(sc)
    net = nrv.Net(c0)
    flat = make_params(c0, seed=9, bias_sigma=0.05)
    net.set_params(torch.from_numpy(flat).to(torch_dev()))
    view = I.fitted_view(sc, 200, 120)
    ds, do = I.depth_normalisation(sc, view)
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    out = torch.empty((120, 200, 3), device=torch_dev())
    nrv.render_batch(scene, net, desc, [view], [out], nrv.PREC_BF16)
    nrv.render_batch(scene, net, desc, [view], [out], nrv.PREC_BF16)   # replayed
    torch.cuda.synchronize()
    _, d, m, g = oracle.rasterize(sc, view)
    xb = oracle.pack(d, m, g, sc.channels, ds, do, 120, 200, 8, 1)       # BF16 input bits
    x = oracle.bf16_value(xb).astype(np.float64)
    ref = unet.forward(x[None, :, :, :c0], unet.unflatten(flat, c0))[0]
    got = out.cpu().numpy()
    assert psnr_range(got, ref) >= 45.0 and np.abs(got - ref).max() <= 2e-2


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_render_batch_groups_views_of_one_size(prec):
    """Views of equal size are shaded by one network call (their images written to each
    caller's buffer); every frame equals the views rendered one at a time through
    nrv_render_batch, captured and replayed alike."""
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.terrain_scene(500, seed=7)
    c0 = len(sc.channels) + 2
    scene = upload_scene(sc)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(make_params(c0, seed=8, bias_sigma=0.05)).to(torch_dev()))
    sizes = [(96, 64), (160, 96), (96, 64), (96, 64), (160, 96)]
    if prec == nrv.PREC_FP8:
        v0 = I.orbit_views(sc, sizes[:1], seed=3)[0]
        xb = torch.zeros((64, 96, 8), dtype=torch.bfloat16, device=torch_dev())
        key = torch.empty((64, 96), dtype=torch.int64, device=torch_dev())
        ds, do = I.depth_normalisation(sc, v0)
        nrv.rasterize(scene, [v0], [key])
        nrv.resolve_pack(scene, v0, key, nrv.make_pack_desc(sc.channels, ds, do), nrv.PREC_BF16, xb)
        net.calibrate(xb, 1, 64, 96)
    outs = [torch.empty((h, w, 3), device=torch_dev()) for (w, h) in sizes]
    single = torch.empty((64, 96, 3), device=torch_dev())
    for frame, seed in enumerate((3, 3, 17)):
        views = I.orbit_views(sc, sizes, seed=seed)
        ds, do = I.depth_normalisation(sc, views[0])
        desc = nrv.make_pack_desc(sc.channels, ds, do)
        nrv.render_batch(scene, net, desc, views, outs, prec)
        torch.cuda.synchronize()
        for v, o in zip(views, outs):
            ref = torch.empty((v.height, v.width, 3), device=torch_dev())
            nrv.render_batch(scene, net, desc, [v], [ref], prec)
            torch.cuda.synchronize()
            assert torch.equal(o, ref), f"frame {frame}: grouped view differs"
    nrv.sync_status()
