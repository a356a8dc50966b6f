"""FP64 oracle of DashGaussian's scheduled densification step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Supplementary "Densification of DashGaussian": at a densification step with
N_GS Gaussians and target P_i, first prune (leaving N'_GS), then clone or
split those Gaussians that meet the backbone's densification condition and
have a top-(P_i - N'_GS) densification score.  The backbone is 3DGS:
score = mean over views of the norm of the view-space (NDC) positional
gradient, condition score >= grad_thresh; prune when opacity < min_opacity
(optionally also when the largest screen radius or world scale is too big);
a selected Gaussian whose largest scale exceeds percent_dense * extent is
split into two samples drawn from it with scales divided by 1.6 (the original
is removed), otherwise it is cloned.

Readings: ties in the top-k are broken by the lower index; appended Gaussians
follow the survivors, in index order of their source (a split source gives its
two samples in sample order); new Gaussians start with zero Adam moments.
Integer decisions are taken in float32 against float32 thresholds (the CUDA
path's precision): score = float32(accum) / float32(count); the opacity test
compares the logit with float32(logit(min_opacity)); the scale tests compare
the largest log-scale with float32(log(threshold)).  Split samples use
mean + R(q) (exp(s) * eps) with eps ~ N(0, I) passed in (noise[j, k]) for
the j-th selected Gaussian in index order.
"""
from __future__ import annotations

import math

import numpy as np


def stats_update(grad_accum, denom, max_radius, grad2d, radius, W, H):
    """Per rendered view: accumulate ||dL/d(ndc)|| = ||(dL/du W/2, dL/dv H/2)||
    for visible Gaussians, their view count and the largest radius."""
    vis = radius > 0
    g = np.hypot(grad2d[:, 0] * (W / 2.0), grad2d[:, 1] * (H / 2.0))
    grad_accum = grad_accum + np.where(vis, g, 0.0)
    denom = denom + vis.astype(np.float64)
    max_radius = np.maximum(max_radius, np.where(vis, radius, 0))
    return grad_accum, denom, max_radius


def thresholds(opts):
    f = np.float32
    return dict(
        grad=f(opts["grad_thresh"]),
        logit_min_opacity=f(math.log(opts["min_opacity"] / (1.0 - opts["min_opacity"]))),
        log_split=f(math.log(opts["percent_dense"] * opts["extent"])),
        max_screen=f(opts.get("max_screen_radius", 0.0)),
        log_max_world=f(math.log(opts["max_world_scale"])) if opts.get("max_world_scale", 0.0) > 0 else None,
    )


def mark(g32, grad_accum32, denom32, max_radius32, opts):
    """Flags of the prune / candidate / split tests (float32 decisions)."""
    t = thresholds(opts)
    logit = g32[:, 10].astype(np.float32)
    lsmax = g32[:, 3:6].astype(np.float32).max(axis=1)
    prune = logit < t["logit_min_opacity"]
    if t["max_screen"] > 0:
        prune |= max_radius32.astype(np.float32) > t["max_screen"]
    if t["log_max_world"] is not None:
        prune |= lsmax > t["log_max_world"]
    keep0 = ~prune
    den = denom32.astype(np.float32)
    with np.errstate(divide="ignore", invalid="ignore"):
        score = np.where(den > 0, grad_accum32.astype(np.float32) / np.where(den > 0, den, np.float32(1)),
                         np.float32(0)).astype(np.float32)
    cand = keep0 & (den > 0) & (score >= t["grad"])
    split = lsmax > t["log_split"]
    return dict(keep0=keep0, cand=cand, split=split, score=score)


def select(cand, score, budget):
    """Top-`budget` candidates by score, ties by lower index; returns a mask."""
    idx = np.nonzero(cand)[0]
    if len(idx) > budget:
        order = sorted(idx.tolist(), key=lambda i: (-float(score[i]), i))
        idx = np.array(sorted(order[:budget]), dtype=np.int64)
    sel = np.zeros(cand.shape, bool)
    sel[idx] = True
    return sel


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def apply(g, m, v, flags, sel, noise):
    """Compaction + appended clones/splits.  g, m, v: (P, 59) FP64.
    Returns (g_new, m_new, v_new)."""
    keep = flags["keep0"] & ~(sel & flags["split"])
    out_g, out_m, out_v = [g[keep]], [m[keep]], [v[keep]]
    sel_idx = np.nonzero(sel)[0]
    new = []
    for j, i in enumerate(sel_idx):
        if flags["split"][i]:
            R = _rot(g[i, 6:10])
            s = np.exp(g[i, 3:6])
            for k in range(2):
                row = g[i].copy()
                row[0:3] = g[i, 0:3] + R @ (s * noise[j, k])
                row[3:6] = g[i, 3:6] - math.log(1.6)
                new.append(row)
        else:
            new.append(g[i].copy())
    if new:
        new = np.array(new)
        out_g.append(new)
        out_m.append(np.zeros_like(new))
        out_v.append(np.zeros_like(new))
    return np.concatenate(out_g), np.concatenate(out_m), np.concatenate(out_v)
