"""Shared test helpers: scene/camera plumbing for the oracle and the CUDA path.

Nothing here computes any part of the rasterizer; it only reshapes seeded
inputs from ``paper_2503_18402_gb300.synth`` into what each side takes.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2503_18402_gb300 import synth


def logit(p):
    return math.log(p / (1.0 - p))


def single_gaussian(mean, log_scale, quat=(1.0, 0.0, 0.0, 0.0), opacity=0.7, dc=(0.8, 0.8, 0.8)):
    """One Gaussian row with only the degree-0 colour term set so that the
    colour (before the +0.5 offset is added back) equals ``dc``."""
    g = np.zeros((1, synth.NPARAM))
    g[0, 0:3] = mean
    g[0, 3:6] = log_scale
    g[0, 6:10] = quat
    g[0, 10] = logit(opacity)
    y00 = 0.5 / math.sqrt(math.pi)
    g[0, 11:14] = (np.asarray(dc, float) - 0.5) / y00
    return g


def identity_cam(width, height, f, cx=None, cy=None):
    vm = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return dict(viewmat=vm, intr=(f, f, width / 2 if cx is None else cx, height / 2 if cy is None else cy),
                width=width, height=height)


def oracle_cam(oracle, cam):
    fx, fy, cx, cy = cam["intr"]
    return oracle.camera(cam["viewmat"], fx, fy, cx, cy, cam["width"], cam["height"])


def cfg0_scene(seed=1000):
    """1,000 Gaussians, one 64x64 camera at distance 4, uniform-random target."""
    g = synth.random_gaussians(1000, seed)
    cam = synth.camera_cfg0(64, 64, 4.0)
    target = synth.target_image(64, 64, seed + 2000)
    return g, cam, target


def _frac_margin(x, tol):
    """True where x is farther than tol from every integer."""
    f = x - np.floor(x)
    return (f > tol) & (f < 1.0 - tol)


def margin_scene(oracle, n, seed, cam, k, tol=1e-4, rel=2e-5, depth_gap=1e-5, max_rounds=20):
    """Float32-representable Gaussians of the 1k-Gaussian recipe, kept only
    where the FP64 projection is away from every discrete threshold of the
    binning, so that FP32 and FP64 arithmetic must give the same tile lists:

      * visible, in front of the near plane by more than tol;
      * u, v farther than tol from an integer (the rect uses floor(u), floor(v));
      * 3 sqrt(lambda_max) farther than tol + rel * value from an integer
        (radius = its ceiling; lambda_max from the FP64 conic);
      * camera depths of any two kept Gaussians apart by more than depth_gap
        relative (the key order is the float32 depth order).

    Rejected Gaussians are redrawn until n are kept.  Returns (g, n_drawn)."""
    rng = np.random.default_rng(seed)
    kept = np.zeros((0, synth.NPARAM))
    drawn = 0
    for _ in range(max_rounds):
        need = n - kept.shape[0]
        if need <= 0:
            break
        cand = synth.random_gaussians(2 * need + 16, int(rng.integers(1 << 31)))
        cand = np.asarray(np.asarray(cand, np.float32), np.float64)
        drawn += cand.shape[0]
        pr = oracle.project(cand, cam, k)
        ok = pr["radius"] > 0
        ok &= pr["depth"] > k.near_plane + tol
        u, v = pr["feat"][:, 0], pr["feat"][:, 1]
        ok &= _frac_margin(u, tol) & _frac_margin(v, tol)
        A, B, C = pr["feat"][:, 2], pr["feat"][:, 3], pr["feat"][:, 4]
        det = A * C - B * B
        with np.errstate(divide="ignore", invalid="ignore"):
            s00, s01, s11 = C / det, -B / det, A / det
            lam = 0.5 * (s00 + s11) + np.sqrt(0.25 * (s00 - s11) ** 2 + s01 ** 2)
            r3 = 3.0 * np.sqrt(lam)
        ok &= np.isfinite(r3) & _frac_margin(r3, tol + rel * np.abs(r3))
        cand, depth = cand[ok], pr["depth"][ok]
        # greedy depth separation against everything kept so far
        keep_depth = list(kept_depth) if kept.shape[0] else []
        sel = []
        for i in np.argsort(rng.uniform(size=cand.shape[0])):
            d = depth[i]
            if all(abs(d - e) > depth_gap * d for e in keep_depth):
                keep_depth.append(d)
                sel.append(i)
            if len(sel) >= need:
                break
        sel = np.sort(np.asarray(sel, np.int64))
        kept = np.concatenate([kept, cand[sel]])
        kept_depth = np.asarray(keep_depth)
    assert kept.shape[0] == n, "margin scene: not enough Gaussians kept"
    return kept, drawn
