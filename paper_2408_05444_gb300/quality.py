"""Image quality of a restoration, as Section 6 reports it (Table 9): PSNR and
SSIM of the restored colour image against the clean one, values in [0, 1].

These are evaluation metrics of the application, computed on the host from the
solver's output; they are not part of the iteration.

SSIM follows Wang, Bovik, Sheikh, Simoncelli, "Image quality assessment: from
error visibility to structural similarity" (IEEE TIP 2004): local means,
variances and covariance under an 11 x 11 Gaussian window of standard deviation
1.5 (normalised to sum 1, evaluated where the window fits inside the image),
constants C1 = (0.01 L)^2 and C2 = (0.03 L)^2 with dynamic range L = 1, the
index averaged over the window positions, and for a colour image averaged over
the three channels.
"""
from __future__ import annotations

import numpy as np


def psnr(x, ref, peak=1.0):
    """10 log10(peak^2 / mean((clip(x, 0, peak) - ref)^2)) in dB."""
    x = np.clip(np.asarray(x, dtype=np.float64), 0.0, peak)
    mse = float(np.mean((x - np.asarray(ref, dtype=np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(peak * peak / mse)


def _window(size=11, sigma=1.5):
    k = np.arange(size) - size // 2
    g = np.exp(-(k ** 2) / (2.0 * sigma ** 2))
    g /= g.sum()
    return g


def _filter_valid(img, g):
    """Separable correlation with the 1-D window g, positions where it fits."""
    s = len(g)
    h, w = img.shape
    rows = sum(g[i] * img[i:h - s + 1 + i, :] for i in range(s))
    return sum(g[j] * rows[:, j:w - s + 1 + j] for j in range(s))


def ssim_channel(x, ref, L=1.0, size=11, sigma=1.5):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(ref, dtype=np.float64)
    if min(x.shape) < size:
        raise ValueError(f"image smaller than the {size} x {size} window")
    g = _window(size, sigma)
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    mx, my = _filter_valid(x, g), _filter_valid(y, g)
    sxx = _filter_valid(x * x, g) - mx * mx
    syy = _filter_valid(y * y, g) - my * my
    sxy = _filter_valid(x * y, g) - mx * my
    num = (2 * mx * my + c1) * (2 * sxy + c2)
    den = (mx * mx + my * my + c1) * (sxx + syy + c2)
    return float(np.mean(num / den))


def ssim(x, ref, L=1.0):
    """Mean SSIM of an h x w (x channels) image, restored values clipped to [0, L]."""
    x = np.clip(np.asarray(x, dtype=np.float64), 0.0, L)
    ref = np.asarray(ref, dtype=np.float64)
    if x.ndim == 2:
        return ssim_channel(x, ref, L)
    return float(np.mean([ssim_channel(x[:, :, c], ref[:, :, c], L) for c in range(x.shape[2])]))
