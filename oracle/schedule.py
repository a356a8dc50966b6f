"""FP64 oracle of DashGaussian's resolution and primitive schedules.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper's steps in its notation:
  * Sec. 4.1: anti-aliased downsampling by r = centre-crop the DFT F to
    (H/r, W/r) and scale it by 1/r^2.  Crop sizes are integers, taken as
    (floor(H/r), floor(W/r)); the crop keeps frequencies
    [-floor(h/2), ceil(h/2) - 1] around DC.
  * Eq. 2: X(F_r) = mean over views of the summed DFT magnitudes of the
    downsampled view.  Reading: the DFT is normalised by the pixel count, so
    the 1/r^2 of Sec. 4.1 (which relates unnormalised transforms) cancels and
    X(r) = sum_{crop(r)} Mbar / (H W), Mbar the view mean of the sum over RGB
    channels of |DFT(I_ch)| (the paper's I has one channel; the channels are
    summed).  With unnormalised transforms X(r) <= X(1)/r^2 for every image,
    so r_m could never exceed sqrt(a) = 2 and the floor modulation would keep
    full resolution throughout, contrary to Sec. 5.3 and the role of a.
  * Sec. 4.2: r_m is where X(F_rm) = X(F)/a (a = 4); X_1..X_{m-1} are
    spaced linearly between X(F) and X(F_rm); r_i solves X(F_ri) = X_i.
    X(r) is a non-increasing step function of r, so "solves" is read as
    r_i = inf{r >= 1 : X(r) <= X_i}, found exactly by walking the intervals
    between crop-size breakpoints (it is always a breakpoint H/n or W/n).  m is not given by the paper; the default
    reading is m = ceil(r_m), capped at 64.
  * Eq. 6/7: anchor s_i = S ln(X_i / X_m) / ln(X_0 / X_m), so s_m = 0 and
    s_0 = S; r equals r_i at iteration s_i and 1/r^2 is linear in k between
    consecutive anchors (Sec. 4.2, last paragraph).
  * Sec. 5 "Implementation Details": the rendering factor is floor(r).
  * Supplementary "Learning Rate": the position learning rate is held at its
    initial value until the first k with floor(r(k)) = 1 and decays from there.
  * Eq. 4: P_k = P_init + (P_fin - P_init) / r^(2 - k/S) with the floored r.
  * Eq. 5: P_fin <- max(P_fin, gamma P_fin + eta P_add), P_fin(0) = 5 P_init,
    gamma = 0.98, eta = 1; updated at each densification step before Eq. 4.
  * Supplementary "Ground Truth Downsampling": downsampling of training views
    is read as area (box) resampling with exact coverage weights.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


MAX_LEVELS = 64  # cap on the number of levels m (reading: m = ceil(r_m), at most 64)


def spectrum_mean(images: np.ndarray) -> np.ndarray:
    """Mbar (H, W): view mean of sum_ch |DFT2(I_ch)|, DC moved to (H//2, W//2)."""
    imgs = np.asarray(images, dtype=np.float64)
    assert imgs.ndim == 4 and imgs.shape[1] == 3
    acc = np.zeros(imgs.shape[2:])
    for n in range(imgs.shape[0]):
        for ch in range(3):
            acc += np.abs(np.fft.fft2(imgs[n, ch]))
    return np.fft.fftshift(acc / imgs.shape[0])


def crop_size(H: int, W: int, r) -> tuple[int, int]:
    """(floor(H/r), floor(W/r)) evaluated exactly (r int, Fraction or float)."""
    r = Fraction(r)
    return int(math.floor(Fraction(H) / r)), int(math.floor(Fraction(W) / r))


def crop_sum(Mbar: np.ndarray, h: int, w: int) -> float:
    H, W = Mbar.shape
    cy, cx = H // 2, W // 2
    return float(Mbar[cy - h // 2: cy + (h + 1) // 2, cx - w // 2: cx + (w + 1) // 2].sum())


def significance(Mbar: np.ndarray, r) -> float:
    """X(F_r) of Eq. 2 for the view-mean magnitude spectrum (pixel-normalised DFT)."""
    H, W = Mbar.shape
    h, w = crop_size(H, W, r)
    return crop_sum(Mbar, h, w) / float(H * W)


def _breakpoints(H: int, W: int) -> list[Fraction]:
    """Values of r > 1 at which floor(H/r) or floor(W/r) drops (exact)."""
    b = {Fraction(H, n) for n in range(1, H)} | {Fraction(W, n) for n in range(1, W)}
    return sorted(x for x in b if x > 1)


def solve_r(Mbar: np.ndarray, target: float) -> float:
    """inf{r >= 1 : X(r) <= target}.  On each interval (lo, hi] between
    consecutive breakpoints the crop is that of hi, so X is constant there and
    the infimum is the left end lo of the first interval where X <= target."""
    H, W = Mbar.shape
    if significance(Mbar, 1) <= target:
        return 1.0
    lo = Fraction(1)
    for hi in _breakpoints(H, W):
        h, w = crop_size(H, W, hi)
        if crop_sum(Mbar, h, w) / float(H * W) <= target:
            return float(lo)
        lo = hi
    return float(lo)  # beyond the last breakpoint the crop is empty


class ResolutionSchedule:
    """Anchors (s_i, r_i) and the per-iteration rendering factor."""

    def __init__(self, Mbar: np.ndarray, S: int, a: float = 4.0, m: int | None = None):
        self.H, self.W = Mbar.shape
        self.S = S
        self.X0 = significance(Mbar, 1)
        self.Xm = self.X0 / a
        self.r_m = solve_r(Mbar, self.Xm)
        self.m = int(math.ceil(self.r_m)) if m is None else int(m)
        self.m = min(max(self.m, 1), MAX_LEVELS)
        self.X = [self.X0 + (i / self.m) * (self.Xm - self.X0) for i in range(self.m + 1)]
        self.r = [1.0] + [solve_r(Mbar, x) for x in self.X[1:]]
        den = math.log(self.X0 / self.Xm)
        self.s = [S * math.log(x / self.Xm) / den for x in self.X]

    def r_cont(self, k: float) -> float:
        """Continuous r(k): 1/r^2 linear in k between consecutive anchors."""
        if k <= self.s[self.m]:
            return self.r[self.m]
        for i in range(self.m, 0, -1):
            s_i, s_prev = self.s[i], self.s[i - 1]
            if k <= s_prev:
                t = (k - s_i) / (s_prev - s_i) if s_prev > s_i else 1.0
                inv2 = (1 - t) / self.r[i] ** 2 + t / self.r[i - 1] ** 2
                return 1.0 / math.sqrt(inv2)
        return self.r[0]

    def r_mod(self, k: float) -> int:
        return max(1, int(math.floor(self.r_cont(k))))

    def render_size(self, k: float) -> tuple[int, int]:
        r = self.r_mod(k)
        return self.H // r, self.W // r

    def first_full_res_iter(self) -> int:
        for k in range(self.S + 1):
            if self.r_mod(k) == 1:
                return k
        return self.S


def position_lr(k: int, k_star: int, S: int, lr_init: float, lr_final: float) -> float:
    """Held at lr_init until k_star, then log-linear decay to lr_final at S."""
    if k <= k_star or S <= k_star:
        return lr_init
    t = min(1.0, (k - k_star) / (S - k_star))
    return math.exp((1 - t) * math.log(lr_init) + t * math.log(lr_final))


def pfin_update(P_fin: float, P_add: float, gamma: float = 0.98, eta: float = 1.0) -> float:
    """Eq. 5."""
    return max(P_fin, gamma * P_fin + eta * P_add)


def primitive_target(k: int, S: int, r_mod: int, P_init: float, P_fin: float) -> float:
    """Eq. 4 with the floored rendering factor."""
    return P_init + (P_fin - P_init) / float(r_mod) ** (2.0 - k / S)


def area_downsample(img: np.ndarray, h: int, w: int) -> np.ndarray:
    """(C, H, W) -> (C, h, w): each output pixel averages the input over its
    footprint [i H/h, (i+1) H/h) x [j W/w, (j+1) W/w) with exact coverage."""
    img = np.asarray(img, dtype=np.float64)
    C, H, W = img.shape

    def weights(n_in, n_out):
        Wm = np.zeros((n_out, n_in))
        for i in range(n_out):
            a, b = Fraction(i * n_in, n_out), Fraction((i + 1) * n_in, n_out)
            for j in range(int(math.floor(a)), int(math.ceil(b))):
                ov = min(b, j + 1) - max(a, j)
                if ov > 0:
                    Wm[i, j] = float(ov / (b - a))
        return Wm
    Wy, Wx = weights(H, h), weights(W, w)
    return np.stack([Wy @ img[c] @ Wx.T for c in range(C)])
