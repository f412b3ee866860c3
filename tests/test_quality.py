"""PSNR / SSIM helpers against closed forms and a window-by-window brute force (CPU)."""
import math

import numpy as np

from paper_2412_11639_gb300 import quality


def test_psnr_closed_form():
    ref = np.zeros((3, 20, 30))
    assert math.isclose(quality.psnr(ref + 0.01, ref), 40.0, rel_tol=1e-12)   # MSE 1e-4
    assert math.isclose(quality.psnr(ref + 0.1, ref, peak=2.0), 10 * math.log10(4 / 0.01), rel_tol=1e-12)
    assert quality.psnr(ref, ref) == float("inf")


def test_ssim_constant_images():
    # zero variance: SSIM = (2ab + C1) / (a^2 + b^2 + C1) at every window
    a, b = 0.3, 0.5
    x = np.full((2, 16, 16), a)
    y = np.full((2, 16, 16), b)
    c1 = 1e-4
    assert math.isclose(quality.ssim(x, y), (2 * a * b + c1) / (a * a + b * b + c1), rel_tol=1e-12)
    assert math.isclose(quality.ssim(x, x), 1.0, rel_tol=1e-12)


def test_ssim_matches_window_bruteforce():
    rng = np.random.default_rng(5)
    x = rng.random((13, 15))
    y = np.clip(x + 0.1 * rng.standard_normal((13, 15)), 0, 1)
    u = np.arange(11) - 5.0
    g = np.exp(-u * u / 4.5)
    w2 = np.outer(g, g) / np.outer(g, g).sum()
    vals = []
    for i in range(13 - 10):
        for j in range(15 - 10):
            px, py = x[i:i + 11, j:j + 11], y[i:i + 11, j:j + 11]
            mx, my = (w2 * px).sum(), (w2 * py).sum()
            vx = (w2 * (px - mx) ** 2).sum()
            vy = (w2 * (py - my) ** 2).sum()
            cxy = (w2 * (px - mx) * (py - my)).sum()
            vals.append(((2 * mx * my + 1e-4) * (2 * cxy + 9e-4)) /
                        ((mx * mx + my * my + 1e-4) * (vx + vy + 9e-4)))
    assert math.isclose(quality.ssim(x, y), float(np.mean(vals)), rel_tol=1e-10)
