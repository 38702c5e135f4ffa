"""PSNR and SSIM (Section 6, Table 9) against their definitions, without a GPU.

SSIM is checked against a brute-force evaluation that visits every window
position with explicit loops over the 11 x 11 Gaussian window (Wang et al.,
IEEE TIP 2004), and against the properties that pin its parts: 1 for identical
images, symmetry, the luminance term alone for constant images, a negative
value for an inverted pattern, and the expected ordering under added noise."""
import numpy as np
import pytest

from paper_2408_05444_gb300 import quality as Q


def _ssim_brute(x, y, L=1.0):
    k = np.arange(11) - 5
    g1 = np.exp(-(k ** 2) / (2 * 1.5 ** 2))
    W = np.outer(g1, g1)
    W /= W.sum()
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    for i in range(x.shape[0] - 10):
        for j in range(x.shape[1] - 10):
            a, b = x[i:i + 11, j:j + 11], y[i:i + 11, j:j + 11]
            ma, mb = np.sum(W * a), np.sum(W * b)
            va = np.sum(W * (a - ma) ** 2)
            vb = np.sum(W * (b - mb) ** 2)
            cab = np.sum(W * (a - ma) * (b - mb))
            vals.append((2 * ma * mb + c1) * (2 * cab + c2) / ((ma ** 2 + mb ** 2 + c1) * (va + vb + c2)))
    return float(np.mean(vals))


def test_ssim_matches_brute_force_windows():
    g = np.random.default_rng(3)
    x = g.random((19, 23))
    y = np.clip(x + 0.1 * g.standard_normal(x.shape), 0, 1)
    assert abs(Q.ssim_channel(x, y) - _ssim_brute(x, y)) < 1e-12
    assert abs(Q.ssim_channel(y, x) - Q.ssim_channel(x, y)) < 1e-14


def test_ssim_properties():
    g = np.random.default_rng(4)
    x = g.random((32, 40, 3))
    assert Q.ssim(x, x) == pytest.approx(1.0, abs=1e-12)
    # constant images: only the luminance term (2 mx my + C1) / (mx^2 + my^2 + C1) remains
    a, b = np.full((16, 16), 0.3), np.full((16, 16), 0.6)
    c1 = 1e-4
    assert Q.ssim_channel(a, b) == pytest.approx((2 * 0.18 + c1) / (0.09 + 0.36 + c1), rel=1e-12)
    # an inverted zero-mean pattern is anti-correlated
    p = 0.5 + 0.4 * np.sign(np.sin(np.arange(32)[:, None] * 0.7) * np.cos(np.arange(32)[None, :] * 0.9))
    assert Q.ssim_channel(p, 1.0 - p) < 0
    # more noise, lower index
    n1 = np.clip(x + 0.02 * g.standard_normal(x.shape), 0, 1)
    n2 = np.clip(x + 0.2 * g.standard_normal(x.shape), 0, 1)
    assert 1.0 > Q.ssim(n1, x) > Q.ssim(n2, x)


def test_psnr_definition():
    x = np.zeros((4, 4))
    ref = np.full((4, 4), 0.1)
    assert Q.psnr(x, ref) == pytest.approx(20.0, abs=1e-12)     # mse 1e-2
    assert Q.psnr(ref, ref) == float("inf")
    assert Q.psnr(np.full((4, 4), 2.0), np.ones((4, 4))) == float("inf")   # clipped to the peak
