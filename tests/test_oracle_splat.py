"""Pins for the Gaussian splat target renderer (stands in for the Gaussian Renderer of
Sec. 4.2): closed forms for one and two Gaussians, the 3-sigma cut-off, early termination,
and invariance to input order."""
import math

import numpy as np

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
