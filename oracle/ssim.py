"""FP64 oracle of the backbone's photometric loss: L1 plus D-SSIM.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the CUDA path.

The paper keeps the 3DGS backbone's optimisation unchanged (Sec. 5,
implementation details), whose training loss is
    L = (1 - lambda) * L1 + lambda * (1 - SSIM),   lambda = 0.2,
with SSIM the structural similarity of Wang et al. 2004 (cited in the
paper's evaluation): local statistics under an 11 x 11 Gaussian window of
standard deviation 1.5 (normalised to sum 1), C1 = 0.01^2, C2 = 0.03^2 for
intensities in [0, 1],
    SSIM(p) = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
averaged over every pixel and channel.  Readings: the window is applied per
channel with zero padding outside the image ("same" size output), and
s_xx = E[x^2] - mu_x^2, s_xy = E[xy] - mu_x mu_y under the window.

The gradient is the exact adjoint: with a = E[x^2] and c = E[xy] (window
sums), SSIM(p) depends on x through mu_x(p), a(p) and c(p), each a window
sum of x, x^2 or x*y, so
    dSSIM/dx(q) = sum_p w(p - q) [dS/dmu_x(p) + 2 x(q) dS/da(p) + y(q) dS/dc(p)],
i.e. the adjoint filter (the same symmetric window, zero padded) applied to
the three per-pixel partial-derivative maps.
"""
from __future__ import annotations

import numpy as np

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """1-D Gaussian window, normalised to sum 1 (the 2-D window is its outer product)."""
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def filter2(img: np.ndarray, w: np.ndarray | None = None) -> np.ndarray:
    """Zero-padded 'same' correlation of every 2-D plane (last two axes)
    with the separable window w x w."""
    w = window() if w is None else w
    r = (len(w) - 1) // 2
    img = np.asarray(img, np.float64)
    H, W = img.shape[-2:]
    pad = np.zeros(img.shape[:-2] + (H, W + 2 * r))
    pad[..., :, r:r + W] = img
    rows = sum(w[k] * pad[..., :, k:k + W] for k in range(len(w)))
    pad = np.zeros(img.shape[:-2] + (H + 2 * r, W))
    pad[..., r:r + H, :] = rows
    return sum(w[k] * pad[..., k:k + H, :] for k in range(len(w)))


def _stats(x, y):
    mu_x, mu_y = filter2(x), filter2(y)
    a, b, c = filter2(x * x), filter2(y * y), filter2(x * y)
    return mu_x, mu_y, a, b, c


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of planar images x, y ([..., H, W], FP64)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mu_x, mu_y, a, b, c = _stats(x, y)
    A1 = 2 * mu_x * mu_y + C1
    A2 = 2 * (c - mu_x * mu_y) + C2
    B1 = mu_x ** 2 + mu_y ** 2 + C1
    B2 = (a - mu_x ** 2) + (b - mu_y ** 2) + C2
    return A1 * A2 / (B1 * B2)


def ssim(x, y) -> float:
    return float(ssim_map(x, y).mean())


def ssim_grad(x, y) -> np.ndarray:
    """d mean(SSIM) / dx, same shape as x."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mu_x, mu_y, a, b, c = _stats(x, y)
    A1 = 2 * mu_x * mu_y + C1
    A2 = 2 * (c - mu_x * mu_y) + C2
    B1 = mu_x ** 2 + mu_y ** 2 + C1
    B2 = (a - mu_x ** 2) + (b - mu_y ** 2) + C2
    S = A1 * A2 / (B1 * B2)
    # partial derivatives of S(mu_x, a, c) with mu_y, b fixed
    dS_dmu = (2 * mu_y * A2 - 2 * mu_y * A1) / (B1 * B2) - S * (2 * mu_x / B1 - 2 * mu_x / B2)
    dS_da = -S / B2
    dS_dc = 2 * A1 / (B1 * B2)
    n = x.size
    return (filter2(dS_dmu) + 2 * x * filter2(dS_da) + y * filter2(dS_dc)) / n


def l1_dssim(x, y, lam: float = LAMBDA):
    """Backbone loss (1 - lam) mean|x - y| + lam (1 - SSIM) of one view and
    its gradient with respect to x (sign(0) = 0 for the L1 term)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    l1 = np.abs(x - y).mean()
    s = ssim(x, y)
    loss = (1 - lam) * l1 + lam * (1 - s)
    grad = (1 - lam) * np.sign(x - y) / n - lam * ssim_grad(x, y)
    return float(loss), grad
