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
