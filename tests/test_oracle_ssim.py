"""Pins of the FP64 L1 + D-SSIM oracle (CPU only).

The window sums are pinned to scipy's Gaussian filter (a library routine);
the SSIM formula to its closed forms (identical images give 1, constant
images give the luminance term alone away from the border) and to a
per-pixel brute-force window sum; the gradient to central finite
differences in FP64.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ssim as S

scipy_nd = pytest.importorskip("scipy.ndimage")


def test_window_sums_match_scipy_gaussian_filter():
    rng = np.random.default_rng(0)
    x = rng.random((3, 20, 23))
    got = S.filter2(x)
    # radius = int(truncate * sigma + 0.5) = 5: the 11-tap window; zero padding
    ref = np.stack([scipy_nd.gaussian_filter(x[c], 1.5, truncate=5 / 1.5, mode="constant", cval=0.0)
                    for c in range(3)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_identical_images_give_one():
    rng = np.random.default_rng(1)
    x = rng.random((3, 17, 12))
    np.testing.assert_allclose(S.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)


def test_constant_images_interior_closed_form():
    a, b = 0.7, 0.2
    x = np.full((1, 30, 31), a)
    y = np.full((1, 30, 31), b)
    m = S.ssim_map(x, y)[0]
    # zero variance and covariance: only the luminance term is left
    expect = (2 * a * b + S.C1) / (a * a + b * b + S.C1)
    np.testing.assert_allclose(m[5:-5, 5:-5], expect, rtol=1e-12)
    # near the border the zero padding lowers the window means: not equal there
    assert abs(m[0, 0] - expect) > 1e-3


def test_symmetric_in_its_arguments():
    rng = np.random.default_rng(2)
    x, y = rng.random((2, 3, 9, 14))
    np.testing.assert_allclose(S.ssim_map(x, y), S.ssim_map(y, x), rtol=1e-13)


def _brute_force_map(x, y):
    """Per-pixel statistics by direct summation over the 11 x 11 window,
    skipping positions outside the image (zero padding)."""
    H, W = x.shape
    w1 = S.window()
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = sxx = syy = sxy = 0.0
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W:
                        wt = w1[di + 5] * w1[dj + 5]
                        mx += wt * x[ii, jj]
                        my += wt * y[ii, jj]
                        sxx += wt * x[ii, jj] ** 2
                        syy += wt * y[ii, jj] ** 2
                        sxy += wt * x[ii, jj] * y[ii, jj]
            vx, vy, cxy = sxx - mx * mx, syy - my * my, sxy - mx * my
            out[i, j] = ((2 * mx * my + S.C1) * (2 * cxy + S.C2)) / ((mx * mx + my * my + S.C1) * (vx + vy + S.C2))
    return out


def test_map_matches_brute_force_window_sums():
    rng = np.random.default_rng(3)
    x, y = rng.random((2, 7, 13))
    np.testing.assert_allclose(S.ssim_map(x[None], y[None])[0], _brute_force_map(x, y), rtol=1e-12, atol=1e-14)


def _fd(f, x, h=1e-6):
    g = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        g[idx] = (f(xp) - f(xm)) / (2 * h)
    return g


def test_ssim_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    x, y = rng.random((2, 2, 8, 13))
    g = S.ssim_grad(x, y)
    fd = _fd(lambda z: S.ssim(z, y), x)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-10)


def test_l1_dssim_loss_and_gradient():
    rng = np.random.default_rng(5)
    x, y = rng.random((2, 3, 6, 9))
    loss, g = S.l1_dssim(x, y)
    assert loss == pytest.approx(0.8 * np.abs(x - y).mean() + 0.2 * (1 - S.ssim(x, y)), rel=1e-14)
    fd = _fd(lambda z: S.l1_dssim(z, y)[0], x)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-10)
    # lambda = 0 is the plain L1 loss
    l0, g0 = S.l1_dssim(x, y, lam=0.0)
    assert l0 == pytest.approx(np.abs(x - y).mean(), rel=1e-14)
    np.testing.assert_array_equal(g0, np.sign(x - y) / x.size)
