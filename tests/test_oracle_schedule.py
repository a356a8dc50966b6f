"""Pins of the FP64 schedule oracle (Sec. 4.1-4.3, Eq. 2, 4, 5, 6, 7, 8)."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import schedule as sch


def _cosine_image(H, W, f, c0, A):
    x = np.arange(W)
    row = c0 + A * np.cos(2 * math.pi * f * x / W)
    img = np.broadcast_to(row[None, :], (H, W))
    return np.stack([img, img, img])[None]


def test_spectrum_mean_matches_direct_dft():
    rng = np.random.default_rng(1)
    imgs = rng.uniform(size=(2, 3, 5, 6))
    H, W = 5, 6
    direct = np.zeros((H, W))
    for n in range(2):
        for ch in range(3):
            for ky in range(H):
                for kx in range(W):
                    s = 0j
                    for y in range(H):
                        for x in range(W):
                            s += imgs[n, ch, y, x] * np.exp(-2j * math.pi * (ky * y / H + kx * x / W))
                    direct[ky, kx] += abs(s) / 2
    # DC moves to (H//2, W//2): frequency k sits at index (k + H//2) mod H
    shifted = np.zeros_like(direct)
    for ky in range(H):
        for kx in range(W):
            shifted[(ky + H // 2) % H, (kx + W // 2) % W] = direct[ky, kx]
    np.testing.assert_allclose(sch.spectrum_mean(imgs), shifted, rtol=1e-12)


def test_constant_image_keeps_all_significance_at_dc():
    # all magnitude at DC: X(r) = X(1) while the crop is non-empty, so X(1)/a is
    # only reached where the crop empties, at r = min(H, W)
    imgs = np.full((1, 3, 32, 48), 0.4)
    Mb = sch.spectrum_mean(imgs)
    assert sch.significance(Mb, 1) == pytest.approx(3 * 0.4, rel=1e-12)  # pixel-normalised DC
    for r in (1.7, 5, 20, 31.9, 32):
        assert sch.significance(Mb, r) == pytest.approx(3 * 0.4, rel=1e-12)
    assert sch.significance(Mb, 32.5) == 0.0
    for a in (4.0, 9.0):
        assert sch.solve_r(Mb, sch.significance(Mb, 1) / a) == 32.0


def _cos_X(W, f, c0, A, r):
    w = math.floor(Fraction(W) / Fraction(r))
    plus = f <= math.ceil(w / 2) - 1
    minus = f <= w // 2
    return 3 * (c0 + 0.5 * A * plus + 0.5 * A * minus)


def test_cosine_image_closed_form_and_jump():
    H, W, f, c0, A = 32, 48, 6, 0.5, 0.3
    Mb = sch.spectrum_mean(_cosine_image(H, W, f, c0, A))
    for r in (1, 1.5, 2, 3.5, Fraction(48, 13), 3.8, 4, 4.2, 6):
        assert sch.significance(Mb, r) == pytest.approx(_cos_X(W, f, c0, A, r), rel=1e-10)
    X0 = sch.significance(Mb, 1)
    # X = 0.8, 0.65 (w = 12) or 0.5 (w <= 11), x3: the first level below X0/1.5 is w <= 11, r > 4
    assert sch.solve_r(Mb, X0 / 1.5) == 4.0
    # X <= 0.7 x3 first holds for w = 12, i.e. r just above 48/13
    assert sch.solve_r(Mb, 3 * 0.7) == pytest.approx(48 / 13, rel=1e-15)
    assert sch.solve_r(Mb, 3 * 0.9) == 1.0


def test_eq7_anchors_by_hand():
    H, W, f, c0, A = 32, 48, 6, 0.5, 0.3
    Mb = sch.spectrum_mean(_cosine_image(H, W, f, c0, A))
    S = 30000
    rs = sch.ResolutionSchedule(Mb, S, a=1.5)
    assert rs.r_m == 4.0 and rs.m == 4
    # X_i = X0 + (i/4)(X0/1.5 - X0) with X0 = 2.4: 2.4, 2.2, 2.0, 1.8, 1.6
    np.testing.assert_allclose(rs.X, [2.4, 2.2, 2.0, 1.8, 1.6], rtol=1e-12)
    # r_i: X <= 2.2 and X <= 2.0 first at w = 12 (X = 1.95): r = 48/13; X <= 1.8 at w = 11: r = 4
    np.testing.assert_allclose(rs.r, [1.0, 48 / 13, 48 / 13, 4.0, 4.0], rtol=1e-15)
    # Eq. 7: s_i = S ln(X_i / X_m) / ln(X_0 / X_m)
    want = [S * math.log(x / 1.6) / math.log(1.5) for x in (2.4, 2.2, 2.0, 1.8, 1.6)]
    np.testing.assert_allclose(rs.s, want, rtol=1e-12, atol=1e-9)
    assert rs.s[0] == pytest.approx(S) and rs.s[4] == pytest.approx(0.0, abs=1e-9)
    # r(k): r_m at k = 0, r_i at s_i, 1/r^2 linear in between
    assert rs.r_cont(0) == 4.0 and rs.r_mod(0) == 4
    assert rs.r_cont(rs.s[1]) == pytest.approx(48 / 13, rel=1e-12)
    k = 0.5 * (rs.s[1] + rs.s[0])
    assert 1 / rs.r_cont(k) ** 2 == pytest.approx(0.5 * (1 + (13 / 48) ** 2), rel=1e-12)
    assert rs.r_cont(S) == pytest.approx(1.0)
    # rendering factor sequence: 4, 3 (once r < 4), 2, 1
    seq = [rs.r_mod(k) for k in range(0, S + 1, 10)]
    assert seq[0] == 4 and seq[-1] == 1 and sorted(set(seq)) == [1, 2, 3, 4]


def test_r_mod_sequence_monotone_and_lr_rule():
    rng = np.random.default_rng(3)
    # a smooth-ish random image with a 1/f spectrum: several levels
    H, W = 48, 64
    ky = np.fft.fftfreq(H)[:, None]; kx = np.fft.fftfreq(W)[None, :]
    amp = 1 / np.maximum(np.hypot(ky, kx), 1 / 64) ** 1.2
    imgs = np.stack([[np.real(np.fft.ifft2(amp * np.exp(2j * math.pi * rng.uniform(size=(H, W)))))
                      for _ in range(3)] for _ in range(2)])
    imgs = imgs - imgs.min() + 0.1
    Mb = sch.spectrum_mean(imgs)
    S = 3000
    rs = sch.ResolutionSchedule(Mb, S, a=4.0)
    seq = [rs.r_mod(k) for k in range(S + 1)]
    assert all(seq[i] >= seq[i + 1] for i in range(S))
    assert seq[0] == max(1, math.floor(rs.r_m)) and seq[-1] == 1
    assert all(rs.s[i] > rs.s[i + 1] for i in range(rs.m))
    ks = rs.first_full_res_iter()
    assert seq[ks] == 1 and (ks == 0 or seq[ks - 1] > 1)
    lr = [sch.position_lr(k, ks, S, 1.6e-4, 1.6e-6) for k in range(S + 1)]
    assert all(v == 1.6e-4 for v in lr[: ks + 1])
    assert lr[-1] == pytest.approx(1.6e-6, rel=1e-12)
    assert all(lr[i] >= lr[i + 1] for i in range(S))


def test_eq5_converges_to_eq8():
    P_add = 1000.0
    for gamma, eta in ((0.98, 1.0), (0.95, 1.0), (0.9, 2.0)):
        P = 10.0
        hist = []
        for _ in range(3000):
            P = sch.pfin_update(P, P_add, gamma, eta)
            hist.append(P)
        assert all(hist[i] <= hist[i + 1] for i in range(len(hist) - 1))  # monotone (max operator)
        assert P == pytest.approx(eta / (1 - gamma) * P_add, rel=1e-9)  # Eq. 8
    # already above the steady state: the max keeps it
    assert sch.pfin_update(1e6, 10.0) == 1e6


def test_eq4_properties():
    S, P0, Pf = 30000, 1e5, 1e6
    assert sch.primitive_target(1234, S, 1, P0, Pf) == Pf  # full resolution: P_k = P_fin
    assert sch.primitive_target(0, S, 4, P0, Pf) == pytest.approx(P0 + (Pf - P0) / 16)
    vals = [sch.primitive_target(k, S, 3, P0, Pf) for k in range(0, S, 100)]
    d1 = np.diff(vals)
    assert np.all(d1 > 0) and np.all(np.diff(d1) > 0)  # increasing and concave-up within a level


def test_area_downsample_pins():
    rng = np.random.default_rng(2)
    img = rng.uniform(size=(3, 12, 18))
    # integer ratio: plain block mean
    out = sch.area_downsample(img, 4, 6)
    np.testing.assert_allclose(out, img.reshape(3, 4, 3, 6, 3).mean(axis=(2, 4)), rtol=1e-13)
    # non-integer ratio: mean preserved, linear ramps sampled at footprint centres
    out = sch.area_downsample(img, 5, 7)
    np.testing.assert_allclose(out.mean(axis=(1, 2)), img.mean(axis=(1, 2)), rtol=1e-12)
    # exact coverage = replicate each pixel h (w) times, then plain block means
    fine = np.repeat(np.repeat(img, 5, axis=1), 7, axis=2)  # (3, 60, 126)
    ref = fine.reshape(3, 5, 12, 7, 18).mean(axis=(2, 4))
    np.testing.assert_allclose(out, ref, rtol=1e-12)
    # constant images stay constant
    np.testing.assert_allclose(sch.area_downsample(np.full((3, 13, 17), 0.3), 4, 9), 0.3, rtol=1e-14)
