"""Image-quality measures of reconstructed frames against a ground-truth intensity.

PSNR with peak 1.0 (intensities are spikes per step for theta = 1) and SSIM after Wang,
Bovik, Sheikh and Simoncelli (IEEE TIP 2004): an 11 x 11 Gaussian window with sigma 1.5,
C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L = 1, averaged over the window positions that lie
inside the frame.  These are host-side evaluation helpers (NumPy), not part of the
reconstruction path.
"""
from __future__ import annotations

import numpy as np


def psnr(x, ref, peak: float = 1.0) -> float:
    """10 log10(peak^2 / MSE) over all elements."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mse = float(np.mean((x - ref) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(peak * peak / mse)


def _gauss(n: int = 11, sigma: float = 1.5) -> np.ndarray:
    u = np.arange(n, dtype=np.float64) - (n - 1) / 2
    g = np.exp(-(u * u) / (2 * sigma * sigma))
    return g / g.sum()


def _filt(a: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Separable 'valid' correlation over the last two axes."""
    n = g.shape[0]
    H, W = a.shape[-2:]
    out = np.zeros(a.shape[:-2] + (H - n + 1, W), dtype=np.float64)
    for i in range(n):
        out += g[i] * a[..., i:i + H - n + 1, :]
    out2 = np.zeros(a.shape[:-2] + (H - n + 1, W - n + 1), dtype=np.float64)
    for i in range(n):
        out2 += g[i] * out[..., :, i:i + W - n + 1]
    return out2


def ssim(x, ref, peak: float = 1.0) -> float:
    """Mean SSIM over frames [..., H, W] (H, W >= 11)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(ref, dtype=np.float64)
    if x.shape != y.shape or x.shape[-1] < 11 or x.shape[-2] < 11:
        raise ValueError("ssim needs equal shapes with H, W >= 11")
    g = _gauss()
    c1, c2 = (0.01 * peak) ** 2, (0.03 * peak) ** 2
    mx, my = _filt(x, g), _filt(y, g)
    sxx = _filt(x * x, g) - mx * mx
    syy = _filt(y * y, g) - my * my
    sxy = _filt(x * y, g) - mx * my
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(s.mean())
