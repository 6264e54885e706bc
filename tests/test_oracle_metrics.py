"""Pins for PSNR and SSIM (Sec. 4.1) against closed forms."""
import math

import numpy as np

from oracle import metrics


def test_psnr_closed_form():
    a = np.zeros((4, 4, 3))
    b = np.full((4, 4, 3), 0.1)
    assert abs(metrics.psnr(a, b) - 20.0) < 1e-12          # MSE 1e-2 -> 20 dB
    assert metrics.psnr(a, a) == math.inf


def test_ssim_identity_and_constants():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (32, 32, 3))
    assert abs(metrics.ssim(x, x) - 1.0) < 1e-12
    a, b = 0.3, 0.7
    c1 = 0.01 ** 2
    # constant images: the structure/contrast term is C2/C2 = 1
    expect = (2 * a * b + c1) / (a * a + b * b + c1)
    got = metrics.ssim(np.full((20, 20), a), np.full((20, 20), b))
    assert abs(got - expect) < 1e-12


def _window_variance(size=11, sigma=1.5):
    """Variance of the offset t - 5 under the normalised 11-tap Gaussian window (sigma 1.5) of
    Wang et al. (2004), from the window's definition."""
    t = np.arange(size) - (size - 1) / 2
    g = np.exp(-t * t / (2 * sigma * sigma))
    g /= g.sum()
    return float((g * t * t).sum())


def test_ssim_scaled_ramp_closed_form():
    """x = a j + b (a ramp along the columns), y = k x.  Under a symmetric window the local
    means are mu_x = a j + b, mu_y = k mu_x; the variances a^2 s^2 and k^2 a^2 s^2 and the
    covariance k a^2 s^2, with s^2 the window's variance along a row.  So per valid position
    SSIM = (2 k mu^2 + C1)(2 k a^2 s^2 + C2) / (((1 + k^2) mu^2 + C1)((1 + k^2) a^2 s^2 + C2)),
    averaged over the columns whose window lies inside the image.  a is chosen so that a^2 s^2
    is comparable to C2: a wrong window width, constant or moment term changes the result."""
    h, w, a, b, k = 24, 40, 0.02, 0.1, 0.5
    j = np.arange(w, dtype=np.float64)
    x = np.tile(a * j + b, (h, 1))
    y = k * x
    s2 = _window_variance()
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    mu = a * j[5:w - 5] + b
    v = a * a * s2
    per = ((2 * k * mu * mu + c1) * (2 * k * v + c2)) / (((1 + k * k) * mu * mu + c1) * ((1 + k * k) * v + c2))
    assert abs(metrics.ssim(x, y) - per.mean()) < 1e-12
    # the same with a window of another width would differ by far more than the tolerance
    assert abs(_window_variance(sigma=1.0) - s2) > 0.5


def test_ssim_brute_force_windows():
    """Every 11 x 11 window of a small random pair, computed directly from its weighted moments
    (no filtering), per channel, averaged."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (16, 18, 2))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    t = np.arange(11) - 5.0
    g1 = np.exp(-t * t / (2 * 1.5 * 1.5))
    g2 = np.outer(g1, g1)
    g2 /= g2.sum()
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    chans = []
    for ch in range(2):
        vals = []
        for i in range(16 - 10):
            for jj in range(18 - 10):
                px = x[i:i + 11, jj:jj + 11, ch]
                py = y[i:i + 11, jj:jj + 11, ch]
                mx, my = (g2 * px).sum(), (g2 * py).sum()
                vx = (g2 * (px - mx) ** 2).sum()
                vy = (g2 * (py - my) ** 2).sum()
                cxy = (g2 * (px - mx) * (py - my)).sum()
                vals.append(((2 * mx * my + c1) * (2 * cxy + c2)) /
                            ((mx * mx + my * my + c1) * (vx + vy + c2)))
        chans.append(np.mean(vals))
    assert abs(metrics.ssim(x, y) - float(np.mean(chans))) < 1e-10
