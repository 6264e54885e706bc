"""VisGlyph (Sec. 4.3, Tab. 2): a masked render pass over the glyph points alone (every 50th
point), which finds per pixel the frontmost glyph point while ignoring the non-glyph points in
front of it.  Keys (carrying the points' indices in the full arrays) and planes bit-exact
against the oracle's render and resolve of that subset, in one call with several views and
through nrv_render_batch."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import make_params, torch_dev

pytestmark = pytest.mark.gpu

S = 50


def _glyph_scene(sc):
    import torch
    from paper_2407_19097_gb300 import nrv
    xyz = torch.from_numpy(np.ascontiguousarray(sc.xyz)).to(torch_dev())
    attr = torch.from_numpy(np.ascontiguousarray(sc.attr).view(np.int32)).to(torch_dev())
    return nrv.Scene(xyz, attr, sc.n_words, point_stride=S)


def _oracle_glyph(sc, view):
    k = oracle.visibility(np.ascontiguousarray(sc.xyz[::S]), view)
    hit = k != np.uint64(0xFFFFFFFFFFFFFFFF)
    j = (k & np.uint64(0xFFFFFFFF)) * np.uint64(S)
    k = np.where(hit, (k & ~np.uint64(0xFFFFFFFF)) | j, k)
    return (k,) + oracle.resolve(k, sc.attr, sc.n_words)


def test_glyph_pass_bit_exact_multi_view():
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.trajectory_scene(20011, 35, seed=2)               # 700k points, 14k glyph points
    views = [I.fitted_view(sc, 320, 200), I.fitted_view(sc, 160, 96, direction=(1, 0.3, 0.2))]
    scene = _glyph_scene(sc)
    keys = [torch.empty((v.height, v.width), dtype=torch.int64, device=torch_dev()) for v in views]
    depth = [torch.empty((v.height, v.width), dtype=torch.int32, device=torch_dev()) for v in views]
    mask = [torch.empty((v.height, v.width), dtype=torch.uint8, device=torch_dev()) for v in views]
    gattr = [torch.empty((sc.n_words, v.height, v.width), dtype=torch.int32, device=torch_dev())
             for v in views]
    nrv.rasterize(scene, views, keys, depth, mask, gattr)
    torch.cuda.synchronize()
    for i, v in enumerate(views):
        rk, rd, rm, rg = _oracle_glyph(sc, v)
        assert np.array_equal(keys[i].cpu().numpy().view(np.uint64), rk)
        assert np.array_equal(depth[i].cpu().numpy().view(np.uint32), rd)
        assert np.array_equal(mask[i].cpu().numpy(), rm)
        assert np.array_equal(gattr[i].cpu().numpy().view(np.uint32), rg)
        # glyph points lie behind or at the frontmost point of the whole cloud
        full = oracle.visibility(sc.xyz, v)
        hit = rk != np.uint64(0xFFFFFFFFFFFFFFFF)
        assert hit.mean() > 0.02
        assert np.all((rk[hit] >> np.uint64(32)) >= (full[hit] >> np.uint64(32)))
        assert np.any((rk[hit] >> np.uint64(32)) > (full[hit] >> np.uint64(32)))


def test_glyph_pass_through_render_batch():
    """The glyph scene shaded end to end: frames equal the glyph keys resolved, packed and
    shaded step by step, captured and replayed alike."""
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.trajectory_scene(20011, 35, seed=2)
    scene = _glyph_scene(sc)
    c0 = len(sc.channels) + 2
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(make_params(c0, seed=3, bias_sigma=0.05)).to(torch_dev()))
    out = torch.empty((96, 160, 3), device=torch_dev())
    for d in ((0, 0, 1), (0, 0, 1), (1, 0.3, 0.2)):
        v = I.fitted_view(sc, 160, 96, direction=d)
        ds, do = I.depth_normalisation(sc, v)
        desc = nrv.make_pack_desc(sc.channels, ds, do)
        nrv.render_batch(scene, net, desc, [v], [out], nrv.PREC_BF16)
        key = torch.empty((96, 160), dtype=torch.int64, device=torch_dev())
        nrv.rasterize(scene, [v], [key])
        xb = torch.empty((96, 160, 8), dtype=torch.bfloat16, device=torch_dev())
        nrv.resolve_pack(scene, v, key, desc, nrv.PREC_BF16, xb)
        ref = torch.empty_like(out)
        net.shade(xb, 1, 96, 160, nrv.PREC_BF16, ref)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        assert np.array_equal(key.cpu().numpy().view(np.uint64), _oracle_glyph(sc, v)[0])
