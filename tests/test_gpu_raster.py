"""GPU parity of the rasterizer (Sec. 3.2): keys and G-buffer planes bit-exact against the CPU
oracle on seeded scenes of every workload family, edge cases included, and packing of the
G-buffer into the network input bit-exact in FP32, BF16 and FP8."""
import numpy as np
import pytest

import nrv_inputs as I
import oracle
from gpu_util import gpu_raster, torch_dev, upload_scene

pytestmark = pytest.mark.gpu


def _check(sc, views, planes=True):
    scene = upload_scene(sc)
    got = gpu_raster(scene, views, planes)
    for v, g in zip(views, got):
        ref = oracle.rasterize(sc, v)
        assert np.array_equal(g[0], ref[0]), f"keys differ in {(g[0] != ref[0]).sum()} pixels"
        if planes:
            for a, b in zip(g[1:], ref[1:]):
                assert np.array_equal(a, b)
    return got


def test_cube_512():
    sc = I.cube_scene(1_000_000, k=3, seed=0)
    _check(sc, [I.cube_view(512, 512)])


def test_vortex_grid_1080p_and_shuffled():
    sc = I.vortex_grid_scene(96, seed=1)
    v = I.cube_view(1920, 1080)
    _check(sc, [v])
    _check(I.shuffled(sc, 5), [v])


def test_trajectories_ragged_sizes():
    sc = I.trajectory_scene(3001, 35, seed=2)          # n = 105035, not a multiple of 4
    views = [I.fitted_view(sc, 1920, 1080), I.fitted_view(sc, 37, 23, direction=(1, 0.3, 0.2))]
    _check(sc, views)


def test_terrain_eight_uneven_views():
    sc = I.terrain_scene(700, seed=7)
    sizes = [(216, 216), (216, 216), (192, 108), (192, 108), (192, 108), (192, 108), (96, 54), (96, 54)]
    views = I.orbit_views(sc, sizes, seed=11, stereo_pairs=1)
    _check(sc, views)


def test_edge_cases(simple_view):
    # empty scene
    sc = I.cube_scene(4, k=3, seed=0)
    empty = I.Scene("empty", sc.xyz[:0].copy(), sc.attr[:0].copy(), 3, sc.channels)
    got = _check(empty, [I.cube_view(33, 17)])
    assert np.all(got[0][0] == np.uint64(0xFFFFFFFFFFFFFFFF))
    # tiny counts around the 4-point grouping, duplicates, clipping, off-screen
    m = [2, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0]
    v = simple_view(m, 8, 4, 0.5, 10.0)
    pts = np.array([[0, 0, 1], [0.25, 0.25, 2], [-0.5, 0.5, 1], [0.5, 0, 1], [0, 0, 0.25],
                    [0.25, 0.25, 2], [0, 0, 0.5], [-0.25, -0.25, 1], [0, 0, 20]], np.float32)
    for n in (1, 2, 3, 5, 7, 9):
        s2 = I.Scene("tiny", pts[:n].copy(), np.arange(4 * n, dtype=np.uint32).reshape(n, 4), 4, [])
        _check(s2, [v])
    # a single-word record stride and a two-word stride
    s1 = I.cube_scene(10_001, k=1, seed=3)
    s1 = I.Scene("k1", s1.xyz, np.ascontiguousarray(s1.attr[:, :1]), 1, s1.channels[:1])
    _check(s1, [I.cube_view(64, 48)])
    s3 = I.terrain_scene(101, seed=7)
    _check(s3, [I.fitted_view(s3, 64, 64, direction=(0.2, 1, 0.1))])


def test_keys_only_mode():
    sc = I.cube_scene(300_000, k=3, seed=9)
    v = I.cube_view(200, 100)
    _check(sc, [v], planes=False)


@pytest.mark.parametrize("prec,cpad", [(0, 8), (1, 8), (2, 16)])
def test_pack_bit_exact(prec, cpad):
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.terrain_scene(500, seed=7)
    v = I.fitted_view(sc, 203, 117, direction=(0.3, 1.0, 0.2))
    scene = upload_scene(sc)
    key, depth, mask, gattr = [None], None, None, None
    dev = torch_dev()
    H, W = v.height, v.width
    keys = [torch.empty((H, W), dtype=torch.int64, device=dev)]
    depth = [torch.empty((H, W), dtype=torch.int32, device=dev)]
    mask = [torch.empty((H, W), dtype=torch.uint8, device=dev)]
    gattr = [torch.empty((2, H, W), dtype=torch.int32, device=dev)]
    nrv.rasterize(scene, [v], keys, depth, mask, gattr)
    ds, do = I.depth_normalisation(sc, v)
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    hn, wn = nrv.lib().nrv_pad8(H), nrv.lib().nrv_pad8(W)
    dt = {0: torch.float32, 1: torch.int16, 2: torch.uint8}[prec]
    netin = torch.empty((hn, wn, cpad), dtype=dt, device=dev)
    inv = 0.37
    nrv.pack(depth[0], mask[0], gattr[0], H, W, desc, prec, netin, inv)
    torch.cuda.synchronize()
    _, od, om, og = oracle.rasterize(sc, v)
    ref = oracle.pack(od, om, og, sc.channels, ds, do, hn, wn, cpad, prec, inv)
    got = netin.cpu().numpy()
    got = got.view(np.uint16) if prec == 1 else got
    assert np.array_equal(got, ref)
    assert (om > 0).mean() > 0.05


def _pinned(i, fn):
    import os
    os.environ["NRV_VIS_VARIANT"] = str(i)
    try:
        return fn()
    finally:
        del os.environ["NRV_VIS_VARIANT"]


def _every_variant(sc, views, scene=None):
    """Keys and planes of every render-pass variant (chunk culling included) equal the oracle's."""
    from paper_2407_19097_gb300 import nrv
    scene = scene or upload_scene(sc)
    refs = [oracle.rasterize(sc, v) for v in views]
    count = nrv.lib().nrv_render_variants(1 if len(views) > 1 else 0)
    assert count >= 2
    for i in range(count):
        got = _pinned(i, lambda: gpu_raster(scene, views))
        for g, ref in zip(got, refs):
            for a, b in zip(g, ref):
                assert np.array_equal(a, b), f"variant {i}: {(a != b).sum()} pixels differ"
    return refs


def test_every_variant_ragged_single_and_multi_view():
    # n = 105035: neither a multiple of 4 nor of the 32-point chunk
    sc = I.trajectory_scene(3001, 35, seed=2)
    views = [I.fitted_view(sc, 1920, 1080), I.fitted_view(sc, 37, 23, direction=(1, 0.3, 0.2))]
    _every_variant(sc, views[:1])
    _every_variant(sc, views)


def test_every_variant_camera_inside_the_cloud():
    # chunks straddle the near plane, lie behind the camera and beyond the far plane
    sc = I.cube_scene(400_003, k=3, seed=4)
    v = I.make_view((0.5, 0.45, 0.52), (0.9, 0.6, 0.1), 640, 480, znear=0.05, zfar=0.6)
    refs = _every_variant(sc, [v])
    assert (refs[0][2] > 0).mean() > 0.05


def test_scene_refresh_after_points_move():
    import dataclasses
    import torch
    from paper_2407_19097_gb300 import nrv
    sc = I.trajectory_scene(20000, 50, seed=3)          # 1M points: chunks mostly hidden
    v = I.fitted_view(sc, 640, 480)
    scene = upload_scene(sc)
    _every_variant(sc, [v], scene)
    # pull every 7th chunk of 32 points halfway towards the camera: hidden chunks become visible
    xyz = sc.xyz.copy()
    eye = np.asarray(v.eye, np.float32)
    idx = np.arange(len(xyz))
    sel = (idx // 32) % 7 == 3
    xyz[sel] = 0.5 * xyz[sel] + 0.5 * eye
    scene.xyz.copy_(torch.from_numpy(xyz).to(scene.xyz.device))
    nrv.check(nrv.lib().nrv_scene_refresh(scene.h))
    _every_variant(dataclasses.replace(sc, xyz=xyz), [v], scene)


def test_partly_visible_chunks_every_variant():
    """One 8-point sub-chunk of every 5th 32-point chunk pulled towards the camera: those
    chunks are visible through one sub-chunk only, so a sub-chunk test that dropped the wrong
    one (or a tile-bound pyramid word below a pixel it covers) would lose keys."""
    import dataclasses
    sc = I.trajectory_scene(20000, 50, seed=5)          # 1M points: chunks mostly hidden
    v = I.fitted_view(sc, 640, 480)
    xyz = sc.xyz.copy()
    eye = np.asarray(v.eye, np.float32)
    idx = np.arange(len(xyz))
    chunk, sub = idx // 32, (idx // 8) % 4
    sel = (chunk % 5 == 2) & (sub == (chunk // 5) % 4)
    xyz[sel] = 0.6 * xyz[sel] + 0.4 * eye
    refs = _every_variant(dataclasses.replace(sc, xyz=xyz), [v])
    # the moved points win a good share of the pixels they reach
    moved = np.isin(refs[0][0] & 0xFFFFFFFF, idx[sel])
    assert moved.sum() > 1000


def test_points_on_pixel_edges_every_variant(simple_view):
    """Points whose projections fall on or within a few ulps of pixel and screen edges, where
    the fast quotient cannot decide the pixel and the exact division must: keys and planes
    bit-exact for every render-pass variant."""
    import os
    from paper_2407_19097_gb300 import nrv
    rng = np.random.default_rng(21)
    W, H, n = 64, 48, 200_003
    m = [2, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0]   # sx = (2x/z + 1) W/2, sy = (1 - 2y/z) H/2
    v = simple_view(m, W, H, 0.5, 10.0)
    z = rng.uniform(1.0, 4.0, n)
    sx = rng.integers(-1, W + 2, n) + rng.choice([0.0, 1e-7, -1e-7, 3e-6, -3e-6, 0.4999], n)
    sy = rng.integers(-1, H + 2, n) + rng.choice([0.0, 2e-7, -2e-7, 5e-6, -5e-6, 0.5], n)
    xyz = np.stack([(sx / (W / 2) - 1) * z / 2, (1 - sy / (H / 2)) * z / 2, z], 1).astype(np.float32)
    base = I.cube_scene(n, k=3, seed=3)
    sc = I.Scene("edges", xyz, base.attr, base.n_words, base.channels)
    scene = upload_scene(sc)
    ref = oracle.rasterize(sc, v)
    assert (ref[2] > 0).mean() > 0.9
    for i in range(nrv.lib().nrv_render_variants(0)):
        os.environ["NRV_VIS_VARIANT"] = str(i)
        try:
            got = gpu_raster(scene, [v])[0]
        finally:
            del os.environ["NRV_VIS_VARIANT"]
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), f"variant {i} differs"
