"""Pins for the oracle's render and resolve passes (Sec. 3.2) against closed forms, brute
force on tiny scenes and invariants -- nothing here re-runs the oracle's own code path."""
import math

import numpy as np
import pytest

import nrv_inputs as I
import oracle
from golden_io import read_raster_case

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def test_golden_closed_form(simple_view):
    m, (w, h, zn, zf), pts, win = read_raster_case()
    view = simple_view(m, w, h, zn, zf)
    key = oracle.visibility(pts, view)
    expect = np.full((h, w), EMPTY, np.uint64)
    for px, py, dbits, idx in win:
        expect[py, px] = np.uint64((dbits << 32) | idx)
    assert np.array_equal(key, expect)


def test_pixel_centres_of_a_pinhole_camera():
    """Points placed on the rays through pixel centres of a 60-degree pinhole camera land on
    those pixels, with depth = distance along the optical axis (geometry, not the matrix)."""
    W, H = 40, 30
    view = I.make_view((0.5, 0.5, 3.0), (0.5, 0.5, 0.5), W, H)
    t = math.tan(math.radians(30.0))
    rng = np.random.default_rng(3)
    pix = [(0, 0), (W - 1, H - 1), (W // 2, H // 2), (W - 1, 0), (0, H - 1)]
    pix += [(int(rng.integers(W)), int(rng.integers(H))) for _ in range(40)]
    pts, depth = [], []
    for k, (px, py) in enumerate(pix):
        D = 1.0 + 0.37 * k
        nx = 2.0 * (px + 0.5) / W - 1.0
        ny = 1.0 - 2.0 * (py + 0.5) / H
        pts.append([0.5 + nx * D * (W / H) * t, 0.5 + ny * D * t, 3.0 - D])
        depth.append(D)
    for k, (px, py) in enumerate(pix):
        key = oracle.visibility(np.array([pts[k]], np.float32), view)
        ys, xs = np.nonzero(key != EMPTY)
        assert (xs.tolist(), ys.tolist()) == ([px], [py])
        d = np.array([int(key[py, px]) >> 32], np.uint32).view(np.float32)[0]
        assert abs(d - depth[k]) <= 1e-5 * depth[k]
        assert int(key[py, px]) & 0xFFFFFFFF == 0


def test_on_axis_point_lands_in_the_centre_pixel():
    view = I.cube_view(512, 512)
    key = oracle.visibility(np.array([[0.5, 0.5, 0.5]], np.float32), view)
    assert key[256, 256] != EMPTY and (key != EMPTY).sum() == 1


def _brute_force(pts, view):
    """O(N * pixels) reference: for each pixel, the (depth, index)-minimum over all points
    whose projection falls in it, compared as tuples (no key packing)."""
    m = np.asarray(view.viewproj, np.float32).reshape(4, 4)
    f = np.float32
    out = {}
    for i, (x, y, z) in enumerate(pts.astype(np.float32)):
        cx = f(f(f(m[0, 0] * x) + f(m[0, 1] * y)) + f(m[0, 2] * z)) + m[0, 3]
        cy = f(f(f(m[1, 0] * x) + f(m[1, 1] * y)) + f(m[1, 2] * z)) + m[1, 3]
        cw = f(f(f(m[3, 0] * x) + f(m[3, 1] * y)) + f(m[3, 2] * z)) + m[3, 3]
        if not (cw >= f(view.znear) and cw <= f(view.zfar)):
            continue
        sx = f(f(cx / cw) + f(1)) * f(0.5 * view.width)
        sy = f(f(1) - f(cy / cw)) * f(0.5 * view.height)
        if not (0 <= sx < view.width and 0 <= sy < view.height):
            continue
        p = (int(sy), int(sx))
        cand = (float(cw), i)
        if p not in out or cand < out[p]:
            out[p] = cand
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tiny_scenes(seed):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.2, 0.8, (64, 3)).astype(np.float32)
    pts[10] = pts[3]          # exact duplicates: lowest index must win
    pts[40] = pts[3]
    view = I.make_view((0.5, 0.5, 2.0), (0.5, 0.5, 0.5), 8, 8)
    key = oracle.visibility(pts, view)
    bf = _brute_force(pts, view)
    for py in range(8):
        for px in range(8):
            k = int(key[py, px])
            if (py, px) in bf:
                d, i = bf[(py, px)]
                assert k & 0xFFFFFFFF == i
                assert np.array([k >> 32], np.uint32).view(np.float32)[0] == np.float32(d)
            else:
                assert k == int(EMPTY)


def test_duplicates_resolve_to_lowest_index(simple_view):
    view = simple_view([2, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0], 8, 4, 0.5, 10.0)
    pts = np.array([[0.1, 0.1, 3.0]] * 5, np.float32)
    key = oracle.visibility(pts, view)
    k = key[key != EMPTY]
    assert k.size == 1 and int(k[0]) & 0xFFFFFFFF == 0
    key2 = oracle.visibility(np.concatenate([np.array([[0.1, 0.1, 4.0]], np.float32), pts]), view)
    assert int(key2[key2 != EMPTY][0]) & 0xFFFFFFFF == 1


def test_depth_plane_invariant_under_permutation():
    sc = I.cube_scene(200_000, k=3, seed=4)
    view = I.cube_view(96, 64)
    d1, m1, _ = oracle.resolve(oracle.visibility(sc.xyz, view), sc.attr, 3)
    perm = np.random.default_rng(8).permutation(sc.n)
    key2 = oracle.visibility(sc.xyz[perm], view)
    d2, m2, _ = oracle.resolve(key2, sc.attr[perm], 3)
    assert np.array_equal(d1, d2) and np.array_equal(m1, m2)
    # the winner's identity maps through the permutation (no exact depth ties here)
    k1 = oracle.visibility(sc.xyz, view)
    hit = k1 != EMPTY
    assert np.array_equal(perm[(key2[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)],
                          (k1[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64))


def test_resolve_copies_the_winners_record():
    sc = I.trajectory_scene(300, 35, seed=5)
    view = I.fitted_view(sc, 64, 48)
    key, depth, mask, gattr = oracle.rasterize(sc, view)
    hit = key != EMPTY
    idx = (key[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.array_equal(depth[hit], (key[hit] >> np.uint64(32)).astype(np.uint32))
    assert np.all(mask[hit] == 1) and np.all(mask[~hit] == 0)
    for c in range(3):
        assert np.array_equal(gattr[c][hit], sc.attr[idx, c])
        assert np.all(gattr[c][~hit] == 0)
    assert np.all(depth[~hit] == 0)
    assert 0.05 < hit.mean() < 1.0


def test_all_core_render_pass_equals_the_sequential_one():
    """The multi-threaded oracle render pass (per-thread minima combined by a minimum) gives the
    sequential pass's keys, ties and duplicates included."""
    import nrv_inputs as I
    sc = I.trajectory_scene(3001, 35, seed=2)
    xyz = np.concatenate([sc.xyz, sc.xyz[::7]])               # duplicates: lowest index wins
    view = I.fitted_view(sc, 200, 120)
    a = oracle.visibility(xyz, view)
    b = oracle.visibility(xyz, view, threads="all")
    assert np.array_equal(a, b)
    assert (a != np.uint64(0xFFFFFFFFFFFFFFFF)).mean() > 0.1
