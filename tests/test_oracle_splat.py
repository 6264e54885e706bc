"""Pins for the Gaussian splat target renderers (they stand in for the Gaussian Renderer of
Sec. 4.2): closed forms for one and two Gaussians, the 3-sigma cut-off, early termination,
invariance to input order, multi-tile binning against unbinned compositing; and for the
anisotropic (velocity-elongated) Gaussians, closed-form screen covariances."""
import math

import numpy as np
import pytest

import oracle

# cx = 2x, cy = 2y, cw = z on a 16 x 16 screen: sx = (2x/z + 1) * 8, sy = (1 - 2y/z) * 8
M = [2, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0]


def _pt(sx, sy, z):
    """World point whose projection is (sx, sy) at depth z on the 16 x 16 test screen."""
    return [(sx / 8.0 - 1.0) * z / 2.0, (1.0 - sy / 8.0) * z / 2.0, z]


def test_single_gaussian_closed_form(simple_view):
    v = simple_view(M, 16, 16, 0.5, 10.0)
    c = np.array([[0.2, 0.5, 1.0]], np.float32)
    img = oracle.splat(np.array([_pt(8.5, 8.5, 1.0)], np.float32), v, c)
    np.testing.assert_allclose(img[8, 8], 0.6 * c[0], rtol=1e-7)
    np.testing.assert_allclose(img[8, 9], 0.6 * math.exp(-1.0 / (2 * 2.25)) * c[0], rtol=1e-7)
    np.testing.assert_allclose(img[10, 11], 0.6 * math.exp(-13.0 / (2 * 2.25)) * c[0], rtol=1e-7)
    assert np.all(img[8, 13] == 0.0)          # 5 px away: beyond 3 sigma = 4.5 px
    assert img[8, 12].sum() > 0.0             # 4 px away: inside


def test_two_gaussians_front_to_back(simple_view):
    v = simple_view(M, 16, 16, 0.5, 10.0)
    c = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], np.float32)
    pts = np.array([_pt(8.5, 8.5, 2.0), _pt(8.5, 8.5, 1.0)], np.float32)   # second is nearer
    img = oracle.splat(pts, v, c)
    np.testing.assert_allclose(img[8, 8], [0.4 * 0.6, 0.6, 0.0], rtol=1e-7)
    img2 = oracle.splat(pts[::-1].copy(), v, c[::-1].copy())
    np.testing.assert_array_equal(img, img2)


def test_transmittance_cut_off(simple_view):
    v = simple_view(M, 16, 16, 0.5, 10.0)
    n = 30
    pts = np.array([_pt(8.5, 8.5, 1.0 + 0.01 * k) for k in range(n)], np.float32)
    c = np.ones((n, 3), np.float32)
    img = oracle.splat(pts, v, c)
    # T_k = 0.4^k; compositing stops after the first k with T < 1e-4, i.e. k = 11
    np.testing.assert_allclose(img[8, 8], 1.0 - 0.4 ** 11, rtol=1e-12)


def test_order_invariance_random(simple_view):
    v = simple_view(M, 16, 16, 0.5, 10.0)
    rng = np.random.default_rng(4)
    pts = np.stack([rng.uniform(-0.6, 0.6, 200), rng.uniform(-0.6, 0.6, 200),
                    rng.uniform(1.0, 2.0, 200)], 1).astype(np.float32)
    c = rng.uniform(0, 1, (200, 3)).astype(np.float32)
    a = oracle.splat(pts, v, c)
    perm = rng.permutation(200)
    b = oracle.splat(pts[perm], v, c[perm])
    np.testing.assert_array_equal(a, b)
    assert a.max() <= 1.0 and a.min() >= 0.0


# ----------------------------------------------------------------- multi-tile screens
# The splatter bins Gaussians into 16 x 16 tiles.  On a 64 x 64 screen (4 x 4 tiles) these pins
# place Gaussians on tile corners, edges and the screen border, so that their 3-sigma discs
# reach one, two or four tiles (or lie partly off screen), and check every pixel of the image.
W64, H48 = 64, 48
M64 = [2, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0]   # sx = (2x/z + 1) W/2, sy = (1 - 2y/z) H/2


def _pt64(sx, sy, z, h=H48):
    """World point projecting to (sx, sy) at depth z on a 64-pixel-wide screen of height h
    (with h = 64, dyadic values are reproduced exactly by the FP32 projection)."""
    return [(sx / 32.0 - 1.0) * z / 2.0, (1.0 - sy / (h / 2.0)) * z / 2.0, z]


def _closed_form_single(sx, sy, colour, h):
    """Image of one Gaussian alone: 0.6 exp(-d^2 / (2 sigma^2)) c within 3 sigma, else 0."""
    py, px = np.mgrid[0:h, 0:W64]
    d2 = (px + 0.5 - sx) ** 2 + (py + 0.5 - sy) ** 2
    a = np.where(d2 <= 4.5 ** 2, 0.6 * np.exp(-d2 / (2 * 1.5 ** 2)), 0.0)
    return a[..., None] * np.asarray(colour, np.float32).astype(np.float64)


# centres: a tile corner (4 tiles), a vertical edge (2 tiles), a horizontal edge, a tile
# interior far from edges (1 tile), a corner of the screen and points off screen whose discs
# still reach it
CENTRES = [(16.0, 16.0), (32.0, 8.5), (40.25, 32.0), (8.0, 40.0), (0.0, 0.0), (-3.5, 20.0),
           (66.0, 63.75), (63.5, 67.0), (47.75, 15.5), (31.875, 48.125), (20.0, 30.0),
           (43.5, 52.0)]


def test_single_gaussians_across_tile_edges(simple_view):
    v = simple_view(M64, W64, 64, 0.5, 10.0)
    c = [0.3, 0.6, 0.9]
    for sx, sy in CENTRES:
        img = oracle.splat(np.array([_pt64(sx, sy, 1.0, 64)], np.float32), v,
                           np.array([c], np.float32))
        np.testing.assert_allclose(img, _closed_form_single(sx, sy, c, 64), rtol=1e-12, atol=0,
                                   err_msg=f"centre {(sx, sy)}")
        assert img.sum() > 0.0


def _project64(xyz):
    """The projection of the splatter (FP32, separate roundings) for the test matrix."""
    x, y, z = (xyz[:, k].astype(np.float32) for k in range(3))
    cx = np.float32(2) * x
    cy = np.float32(2) * y
    cw = z
    sx = (cx / cw + np.float32(1)) * np.float32(32)
    sy = (np.float32(1) - cy / cw) * np.float32(24)
    return cw, sx.astype(np.float64), sy.astype(np.float64)


def _brute_force_splat(xyz, colour, znear, zfar):
    """Unbinned compositing: every pixel walks the whole list sorted by (w, index)."""
    cw, sx, sy = _project64(xyz)
    keep = [i for i in range(len(cw)) if znear <= cw[i] <= zfar and -4.5 <= sx[i] < W64 + 4.5
            and -4.5 <= sy[i] < H48 + 4.5]
    order = sorted(keep, key=lambda i: (float(cw[i]), i))
    out = np.zeros((H48, W64, 3))
    for py in range(H48):
        for px in range(W64):
            cx, cy, tr = px + 0.5, py + 0.5, 1.0
            acc = [0.0, 0.0, 0.0]
            for i in order:
                dx, dy = cx - sx[i], cy - sy[i]
                d2 = dx * dx + dy * dy
                if d2 > 4.5 * 4.5:
                    continue
                a = 0.6 * math.exp(-d2 / (2.0 * 1.5 * 1.5))
                for j in range(3):
                    acc[j] += tr * a * float(colour[i, j])
                tr *= 1.0 - a
                if tr < 1e-4:
                    break
            out[py, px] = acc
    return out


def test_random_multi_tile_scene_matches_unbinned_loop(simple_view):
    v = simple_view(M64, W64, H48, 0.5, 10.0)
    rng = np.random.default_rng(11)
    n = 160
    sx = rng.uniform(-6.0, W64 + 6.0, n)
    sy = rng.uniform(-6.0, H48 + 6.0, n)
    z = rng.uniform(0.4, 3.0, n)                       # some in front of the near plane
    pts = np.array([_pt64(a, b, c) for a, b, c in zip(sx, sy, z)], np.float32)
    # a few exact depth ties: the lower index goes first
    pts[10:14, 2] = pts[9, 2]
    colour = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    got = oracle.splat(pts, v, colour)
    want = _brute_force_splat(pts, colour, 0.5, 10.0)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
    assert (got.sum(axis=2) > 0).mean() > 0.5          # the scene covers most tiles


def test_many_points_match_a_per_pixel_reference(simple_view):
    """50k Gaussians on a 96 x 80 screen (30 tiles), enough for every thread of the splatter's
    parallel filter, sort and binning to hold many points: each pixel against a reference that
    sorts all covering Gaussians by (w, index) with numpy and composites them in that order."""
    W, H = 96, 80
    m = [2, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0]
    v = simple_view(m, W, H, 0.5, 10.0)
    rng = np.random.default_rng(12)
    n = 50_000
    sx = rng.uniform(-6.0, W + 6.0, n)
    sy = rng.uniform(-6.0, H + 6.0, n)
    z = rng.choice(np.linspace(0.4, 3.0, 4000), n)          # many exact depth ties
    pts = np.stack([(sx / (W / 2) - 1) * z / 2, (1 - sy / (H / 2)) * z / 2, z], 1).astype(np.float32)
    colour = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    got = oracle.splat(pts, v, colour)
    x, y, zz = (pts[:, k].astype(np.float32) for k in range(3))
    cw = zz
    px = ((np.float32(2) * x / cw + np.float32(1)) * np.float32(W / 2)).astype(np.float64)
    py = ((np.float32(1) - np.float32(2) * y / cw) * np.float32(H / 2)).astype(np.float64)
    keep = (cw >= np.float32(0.5)) & (cw <= np.float32(10.0)) & (px >= -4.5) & (px < W + 4.5) & \
        (py >= -4.5) & (py < H + 4.5)
    idx = np.nonzero(keep)[0]
    order = idx[np.lexsort((idx, cw[idx]))]                   # by w, then index
    ox, oy, oc = px[order], py[order], colour[order].astype(np.float64)
    want = np.zeros((H, W, 3))
    for yy in range(H):
        for xx in range(W):
            d2 = (xx + 0.5 - ox) ** 2 + (yy + 0.5 - oy) ** 2
            sel = np.nonzero(d2 <= 4.5 * 4.5)[0]
            tr, acc = 1.0, np.zeros(3)
            for k in sel:
                a = 0.6 * math.exp(-d2[k] / (2.0 * 1.5 * 1.5))
                acc += tr * a * oc[k]
                tr *= 1.0 - a
                if tr < 1e-4:
                    break
            want[yy, xx] = acc
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


# ----------------------------------------------------------------- anisotropic Gaussians
# On the 64 x 64 screen (cx = 2x, cy = 2y, cw = z) a point on the axis at depth 1 has the
# screen-map Jacobian J = [[64, 0, 0], [0, -64, 0]], so a velocity along x gives the screen
# covariance diag((64 r0 s)^2, (64 r0)^2); r0 = 1.5 / 64 makes the short axis 1.5 px.
R0 = 1.5 / 64.0


def _aniso_closed_form(sx, sy, cov, colour):
    py, px = np.mgrid[0:64, 0:64]
    dx, dy = px + 0.5 - sx, py + 0.5 - sy
    a, b, c = cov
    det = a * c - b * b
    q = (c * dx * dx - 2 * b * dx * dy + a * dy * dy) / det
    inside = (q <= 9.0) & (np.abs(dx) <= 3 * np.sqrt(a)) & (np.abs(dy) <= 3 * np.sqrt(c))
    al = np.where(inside, 0.6 * np.exp(-0.5 * q), 0.0)
    return al[..., None] * np.asarray(colour, np.float32).astype(np.float64)


@pytest.mark.parametrize("stretch", [1.0, 3.0, 6.0])
def test_aniso_single_gaussian_along_x(simple_view, stretch):
    v = simple_view(M64, 64, 64, 0.5, 10.0)
    p = np.array([[0.0, 0.0, 1.0]], np.float32)            # projects to (32, 32)
    col = [[0.2, 0.7, 0.4]]
    img = oracle.splat_aniso(p, v, np.array(col, np.float32), np.array([[2.5, 0, 0]], np.float32),
                             R0, stretch)
    cov = ((64 * R0 * stretch) ** 2, 0.0, (64 * R0) ** 2)
    np.testing.assert_allclose(img, _aniso_closed_form(32.0, 32.0, cov, col[0]), rtol=1e-12, atol=1e-15)
    if stretch == 1.0:   # the isotropic renderer with sigma = 1.5 px
        iso = oracle.splat(p, v, np.array(col, np.float32))
        np.testing.assert_allclose(img, iso, rtol=1e-12, atol=1e-15)


def test_aniso_diagonal_velocity_and_zero_velocity(simple_view):
    """A velocity along (1, 1, 0) (screen y points down, so the long axis is (1, -1)) and a point
    without velocity (isotropic), each against its closed-form covariance."""
    v = simple_view(M64, 64, 64, 0.5, 10.0)
    p = np.array([[0.0, 0.0, 1.0]], np.float32)
    col = [[1.0, 0.5, 0.25]]
    s = 4.0
    img = oracle.splat_aniso(p, v, np.array(col, np.float32), np.array([[1, 1, 0]], np.float32), R0, s)
    u = np.array([1.0, -1.0]) / np.sqrt(2.0)
    cov2 = (64 * R0) ** 2 * (np.eye(2) + (s * s - 1) * np.outer(u, u))
    np.testing.assert_allclose(img, _aniso_closed_form(32.0, 32.0, (cov2[0, 0], cov2[0, 1], cov2[1, 1]), col[0]),
                               rtol=1e-10, atol=1e-14)
    img0 = oracle.splat_aniso(p, v, np.array(col, np.float32), np.zeros((1, 3), np.float32), R0, s)
    np.testing.assert_allclose(img0, oracle.splat(p, v, np.array(col, np.float32)), rtol=1e-12, atol=1e-15)


def test_aniso_depth_scaling_and_order(simple_view):
    """At depth z the Jacobian scales by 1/z (the footprint shrinks), nearer points composite
    first whatever the input order."""
    v = simple_view(M64, 64, 64, 0.5, 10.0)
    col = np.array([[1, 0, 0], [0, 1, 0]], np.float32)
    vel = np.array([[1, 0, 0], [0, 1, 0]], np.float32)
    pts = np.array([[0.0, 0.0, 2.0], [0.0, 0.0, 1.0]], np.float32)   # the second is nearer
    img = oracle.splat_aniso(pts, v, col, vel, R0, 3.0)
    img2 = oracle.splat_aniso(pts[::-1].copy(), v, col[::-1].copy(), vel[::-1].copy(), R0, 3.0)
    np.testing.assert_array_equal(img, img2)
    # centre pixel: the near Gaussian (alpha 0.6 at its centre offset) over the far one
    near = _aniso_closed_form(32.0, 32.0, ((64 * R0) ** 2, 0.0, (64 * R0 * 3) ** 2), [0, 1, 0])
    far = _aniso_closed_form(32.0, 32.0, ((32 * R0 * 3) ** 2, 0.0, (32 * R0) ** 2), [1, 0, 0])
    a_near = near[..., 1]
    np.testing.assert_allclose(img[..., 1], a_near, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(img[..., 0], (1 - a_near) * far[..., 0], rtol=1e-12, atol=1e-15)
