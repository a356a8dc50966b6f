"""Pins of the densification oracle (supplementary "Densification of
DashGaussian"; the 3DGS clone/split routine it keeps)."""
from __future__ import annotations

import math

import numpy as np

from oracle import densify as D
from paper_2503_18402_gb300 import synth

OPTS = dict(grad_thresh=2e-4, min_opacity=0.005, percent_dense=0.01, extent=5.0)


def _state(n, seed):
    rng = np.random.default_rng(seed)
    g = synth.random_gaussians(n, seed)
    g[:, 10] = rng.normal(-3.0, 2.5, size=n)  # some below the opacity threshold
    g[:, 3:6] = rng.normal(-3.9, 0.4, size=(n, 3))  # split threshold log(0.05) = -3.0
    acc = np.abs(rng.normal(0, 6e-4, size=n)) * 3
    den = rng.integers(0, 4, size=n).astype(np.float64)
    acc[den == 0] = 0
    return g, acc, den


def test_stats_closed_form():
    g2 = np.zeros((3, 9)); g2[:, 0] = [1e-4, 2e-4, 0.0]; g2[:, 1] = [3e-4, 0.0, 5e-4]
    acc, den, mr = D.stats_update(np.zeros(3), np.zeros(3), np.zeros(3), g2, np.array([4, 0, 7]), 100, 60)
    np.testing.assert_allclose(acc, [math.hypot(1e-4 * 50, 3e-4 * 30), 0.0, math.hypot(0, 5e-4 * 30)])
    np.testing.assert_array_equal(den, [1, 0, 1])
    np.testing.assert_array_equal(mr, [4, 0, 7])


def test_mark_matches_plain_definitions():
    g, acc, den = _state(3000, 1)
    f = D.mark(g.astype(np.float32), acc.astype(np.float32), den.astype(np.float32), np.zeros(3000, np.float32), OPTS)
    o = 1 / (1 + np.exp(-g[:, 10].astype(np.float32).astype(np.float64)))
    far = np.abs(o - 0.005) > 1e-6  # away from the decision boundary both definitions agree
    np.testing.assert_array_equal(f["keep0"][far], (o >= 0.005)[far])
    score = np.where(den > 0, acc / np.maximum(den, 1), 0)
    ok = np.abs(score - 2e-4) > 1e-9
    np.testing.assert_array_equal(f["cand"][ok], (f["keep0"] & (den > 0) & (score >= 2e-4))[ok])
    smax = np.exp(g[:, 3:6]).max(1)
    ok = np.abs(smax - 0.05) > 1e-7
    np.testing.assert_array_equal(f["split"][ok], (smax > 0.05)[ok])
    assert f["keep0"].sum() < 3000 and f["cand"].sum() > 100 and f["split"].sum() > 50


def test_topk_selection_against_lexsort():
    rng = np.random.default_rng(3)
    cand = rng.uniform(size=500) < 0.6
    score = rng.integers(0, 40, size=500).astype(np.float32)  # many ties
    for budget in (0, 1, 17, 250, 1000):
        sel = D.select(cand, score, budget)
        idx = np.nonzero(cand)[0]
        order = idx[np.lexsort((idx, -score[idx]))]
        np.testing.assert_array_equal(np.nonzero(sel)[0], np.sort(order[:budget]))


def test_apply_counts_order_and_samples():
    g, acc, den = _state(2000, 4)
    m = np.random.default_rng(5).normal(size=g.shape)
    v = np.abs(m)
    f = D.mark(g.astype(np.float32), acc.astype(np.float32), den.astype(np.float32), np.zeros(2000, np.float32), OPTS)
    budget = int(f["cand"].sum() // 2)
    sel = D.select(f["cand"], f["score"], budget)
    noise = np.zeros((budget, 2, 3))
    g2, m2, v2 = D.apply(g, m, v, f, sel, noise)
    n_keep0 = int(f["keep0"].sum())
    assert g2.shape[0] == n_keep0 + int(sel.sum())
    keep = f["keep0"] & ~(sel & f["split"])
    np.testing.assert_array_equal(g2[: keep.sum()], g[keep])
    np.testing.assert_array_equal(m2[: keep.sum()], m[keep])
    new = g2[keep.sum():]
    assert np.all(m2[keep.sum():] == 0) and np.all(v2[keep.sum():] == 0)
    # zero noise: split samples sit on the mean with scale / 1.6; clones are copies
    r = 0
    for i in np.nonzero(sel)[0]:
        if f["split"][i]:
            for _ in range(2):
                np.testing.assert_allclose(new[r, 0:3], g[i, 0:3], atol=1e-15)
                np.testing.assert_allclose(np.exp(new[r, 3:6]), np.exp(g[i, 3:6]) / 1.6, rtol=1e-14)
                np.testing.assert_array_equal(new[r, 6:], g[i, 6:])
                r += 1
        else:
            np.testing.assert_array_equal(new[r], g[i])
            r += 1
    assert r == new.shape[0]


def test_split_samples_follow_the_gaussian():
    # the empirical covariance of many split samples approaches Sigma = R S^2 R^T
    g = synth.random_gaussians(1, 9)
    g[0, 3:6] = np.log([0.3, 0.1, 0.05])
    rng = np.random.default_rng(0)
    n = 20000
    flags = dict(keep0=np.ones(n, bool), split=np.ones(n, bool))
    gg = np.repeat(g, n, axis=0)
    noise = rng.normal(size=(n, 2, 3))
    g2, _, _ = D.apply(gg, gg * 0, gg * 0, flags, np.ones(n, bool), noise)
    pts = g2[:, 0:3] - g[0, 0:3]
    q = g[0, 6:10] / np.linalg.norm(g[0, 6:10])
    from scipy.spatial.transform import Rotation
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sigma = R @ np.diag([0.3, 0.1, 0.05]) ** 2 @ R.T
    np.testing.assert_allclose(np.cov(pts.T), Sigma, atol=3e-3 * 0.09)
