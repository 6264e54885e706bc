"""CPU ORACLE (test infrastructure only): image quality metrics used by the paper (Sec. 4.1).

PSNR = 10 log10(R^2 / MSE) over all pixels and channels.  SSIM follows Wang et al. (2004):
per channel, local statistics under an 11x11 Gaussian window with sigma 1.5 (only windows
fully inside the image), C1 = (0.01 R)^2, C2 = (0.03 R)^2, averaged over positions and then
over channels.  The Gaussian filtering uses scipy's 1-D correlation as a library primitive.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate1d


def psnr(a, b, data_range: float = 1.0) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    mse = float(np.mean((a - b) ** 2))
    if mse == 0.0:
        return float("inf")
    return 10.0 * np.log10(data_range * data_range / mse)


def _gauss_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _filter_valid(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    r = len(g) // 2
    f = correlate1d(correlate1d(img, g, axis=0, mode="constant"), g, axis=1, mode="constant")
    return f[r:img.shape[0] - r, r:img.shape[1] - r]


def ssim(a, b, data_range: float = 1.0) -> float:
    """Mean SSIM of two HxWxC (or HxW) images."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.ndim == 2:
        a, b = a[..., None], b[..., None]
    g = _gauss_window()
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    vals = []
    for ch in range(a.shape[-1]):
        x, y = a[..., ch], b[..., ch]
        mx, my = _filter_valid(x, g), _filter_valid(y, g)
        sxx = _filter_valid(x * x, g) - mx * mx
        syy = _filter_valid(y * y, g) - my * my
        sxy = _filter_valid(x * y, g) - mx * my
        m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        vals.append(float(m.mean()))
    return float(np.mean(vals))
