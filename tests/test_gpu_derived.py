"""Derived channels of the resolve pass (Sec. 4.5 Vel2D, Sec. 3.2 splat radius) against the
FP64 oracle: nrv_resolve_pack on a vortex-grid frame, FP32 output, every derived format next to
a plain channel; and nrv_render_batch with derived channels, captured and replayed with moved
cameras, bit-identical to the step-by-step path."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import make_params, torch_dev, upload_scene

pytestmark = pytest.mark.gpu

DERIVED = [oracle.VEL2D_X, oracle.VEL2D_Y, oracle.VEL2D_ANGLE, oracle.VEL2D_MAG, oracle.SPLAT_RADIUS]


def _desc(sc, view):
    from paper_2407_19097_gb300 import nrv
    ch = [I.Channel(0, f) for f in DERIVED[:4]] + [I.Channel(3, oracle.SPLAT_RADIUS), I.Channel(4, 0)]
    ds, do = I.depth_normalisation(sc, view)
    return ch, ds, do, nrv.make_pack_desc(ch, ds, do)


def test_resolve_pack_derived_channels_vs_oracle():
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.vortex_grid_scene(64, seed=1)           # record: v (3), |v|, pressure
    view = I.make_view((0.2, 0.8, 2.2), (0.5, 0.5, 0.5), 320, 200)
    scene = upload_scene(sc)
    H, W = view.height, view.width
    key = torch.empty((H, W), dtype=torch.int64, device=torch_dev())
    nrv.rasterize(scene, [view], [key])
    ch, ds, do, desc = _desc(sc, view)
    hn, wn = nrv.lib().nrv_pad8(H), nrv.lib().nrv_pad8(W)
    netin = torch.empty((hn, wn, 8), dtype=torch.float32, device=torch_dev())
    nrv.resolve_pack(scene, view, key, desc, nrv.PREC_F32, netin)
    torch.cuda.synchronize()
    got = netin.cpu().numpy()
    k = key.cpu().numpy().view(np.uint64)
    ref_key = oracle.visibility(sc.xyz, view)
    assert np.array_equal(k, ref_key)
    hit = k != np.uint64(0xFFFFFFFFFFFFFFFF)
    assert hit.mean() > 0.2
    # the plain channel, depth and coverage: bit-exact with the oracle's pack
    _, d, m, g = oracle.rasterize(sc, view)
    plain = oracle.pack(d, m, g, [ch[5]], ds, do, hn, wn, 8, 0)
    np.testing.assert_array_equal(got[..., 5], plain[..., 0])
    np.testing.assert_array_equal(got[..., 6:8], plain[..., 1:3])
    for j, c in enumerate(ch[:5]):
        ref = oracle.derived_channel(k, sc.xyz, sc.attr, view, c.fmt, c.word)
        g = got[:H, :W, j].astype(np.float64)
        assert np.all(g[~hit] == 0.0)
        r, gv = ref[hit], g[hit]
        if c.fmt == oracle.VEL2D_ANGLE:
            mag = oracle.derived_channel(k, sc.xyz, sc.attr, view, oracle.VEL2D_MAG, 0)[hit]
            ok = mag > 1e-3 * np.median(mag)           # the angle of a vanishing v' is unstable
            d = np.abs(np.angle(np.exp(1j * (gv[ok] - r[ok]))))
            assert d.max() <= 1e-4, (c.fmt, d.max())
        else:
            scale = np.sqrt(np.mean(r * r))
            err = np.abs(gv - r) / (np.abs(r) + scale)
            assert err.max() <= 2e-5, (c.fmt, err.max())
    # the G-buffer-plane pack refuses derived formats
    with pytest.raises(nrv.NrvError):
        depth = torch.empty((H, W), dtype=torch.int32, device=torch_dev())
        mask = torch.empty((H, W), dtype=torch.uint8, device=torch_dev())
        gat = torch.empty((sc.n_words, H, W), dtype=torch.int32, device=torch_dev())
        nrv.pack(depth, mask, gat, H, W, desc, nrv.PREC_F32, netin)


def test_render_batch_derived_channels_replay():
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.vortex_grid_scene(48, seed=2)
    scene = upload_scene(sc)
    c0 = 8
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(make_params(c0, seed=6, bias_sigma=0.05)).to(torch_dev()))
    sizes = [(160, 96), (96, 64)]
    outs = [torch.empty((h, w, 3), device=torch_dev()) for (w, h) in sizes]
    for frame, eye in enumerate([(0.2, 0.8, 2.2), (0.2, 0.8, 2.2), (1.5, 0.6, 1.9), (-0.4, 1.1, 1.6)]):
        views = [I.make_view(eye, (0.5, 0.5, 0.5), w, h) for (w, h) in sizes]
        ch, ds, do, desc = _desc(sc, views[0])
        nrv.render_batch(scene, net, desc, views, outs, nrv.PREC_BF16)
        torch.cuda.synchronize()
        for v, o in zip(views, outs):
            H, W = v.height, v.width
            key = torch.empty((H, W), dtype=torch.int64, device=torch_dev())
            nrv.rasterize(scene, [v], [key])
            xb = torch.empty((nrv.lib().nrv_pad8(H), nrv.lib().nrv_pad8(W), 8), dtype=torch.bfloat16,
                             device=torch_dev())
            nrv.resolve_pack(scene, v, key, desc, nrv.PREC_BF16, xb)
            ref = torch.empty((H, W, 3), device=torch_dev())
            net.shade(xb, 1, H, W, nrv.PREC_BF16, ref)
            torch.cuda.synchronize()
            assert torch.equal(o, ref), f"frame {frame}: batch differs from step by step"
