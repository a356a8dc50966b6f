"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module draws scenes, cameras and target images only; it contains none of
the rasterizer's or the schedule's arithmetic, so that both implementations
can consume identical inputs without sharing any of the method's code.

Per-Gaussian parameter row (59 values), the interface both sides use:
    0:3   mean (world)            3:6   log scale
    6:10  quaternion (w, x, y, z) 10    opacity logit
    11:59 SH coefficients, coefficient-major: 11 + 3*k + channel, k = l*l + l + m

Scene recipes (the paper evaluates on Mip-NeRF 360, Deep Blending and
Tanks&Temples, which are not available here; these seeded scenes stand in for
them with the shapes and parameter distributions of the workloads):
  * ``random_gaussians``: means U[-1,1]^3, log-scales N(-3, 0.5), random unit
    quaternions, opacity logit N(0, 1), SH coefficients N(0, 0.2^2).
  * ``textured_scene``: a dead-leaves layout (the classic model of
    natural-image statistics): 400 plane patches and spheres with half-sizes
    from the scale-invariant density p(s) ~ s^-3 on [0.04, 0.9], placed in
    [-1.8, 1.8]^3, each with its own base colour and a seeded texture with a
    1/f amplitude spectrum (32 plane waves, 0.5 to 40 cycles per unit of
    surface coordinate) setting the SH DC colour; 90% of the Gaussians spread
    over the surfaces in proportion to area, 10% on a background shell of
    radius 12.  Each Gaussian's scale is the local spacing sqrt(area / count)
    with a log-normal spread (std 0.3), so surfaces are closed and resolved
    down to the Gaussian spacing (about a pixel at 1237x822 for 2M
    Gaussians); quaternions, opacity logits and higher SH are drawn as in
    ``random_gaussians``.
"""
from __future__ import annotations

import math

import numpy as np

NPARAM = 59
SH_DC_NORM = 0.28209479177387814  # value of the degree-0 basis, used only to pick DC colours


def random_gaussians(n: int, seed: int, extent: float = 1.0) -> np.ndarray:
    """(n, 59) float64 Gaussians with the distributions of the 1k-Gaussian scene."""
    rng = np.random.default_rng(seed)
    g = np.zeros((n, NPARAM))
    g[:, 0:3] = rng.uniform(-extent, extent, size=(n, 3))
    g[:, 3:6] = rng.normal(-3.0, 0.5, size=(n, 3))
    q = rng.normal(size=(n, 4))
    g[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True)
    g[:, 10] = rng.normal(0.0, 1.0, size=n)
    g[:, 11:59] = rng.normal(0.0, 0.2, size=(n, 48))
    return g


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World-to-camera [R|t] (3x4) of a camera at ``eye`` looking at ``target``
    (x right, y down, z forward)."""
    eye = np.asarray(eye, float)
    fwd = np.asarray(target, float) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, float))
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])  # rows: camera axes in world coordinates
    t = -R @ eye
    return np.concatenate([R, t[:, None]], axis=1)


def intrinsics(width: int, height: int, fov_x_deg: float = 60.0):
    """(fx, fy, cx, cy) of a pinhole with square pixels and centred principal point."""
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return fx, fx, 0.5 * width, 0.5 * height


def camera_cfg0(width: int = 64, height: int = 64, distance: float = 4.0):
    eye = np.array([distance * 0.6, -distance * 0.64, distance * 0.48])
    eye *= distance / np.linalg.norm(eye)
    return dict(viewmat=look_at(eye), intr=intrinsics(width, height), width=width, height=height)


def ring_cameras(n_views: int, width: int, height: int, radius: float, seed: int):
    """Views on a hemisphere ring band around the origin, all looking at it."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n_views):
        az = 2.0 * math.pi * (i + rng.uniform(-0.3, 0.3)) / n_views
        el = math.radians(rng.uniform(5.0, 50.0))
        eye = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams.append(dict(viewmat=look_at(eye), intr=intrinsics(width, height),
                         width=width, height=height))
    return cams


def target_image(width: int, height: int, seed: int) -> np.ndarray:
    """(3, H, W) uniform random target image."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(3, height, width))


def _band_noise(rng, n_waves=32, f_lo=0.5, f_hi=40.0, std=0.25):
    """Texture over surface coordinates with a natural-image-like 1/f
    amplitude spectrum: plane waves with log-uniform spatial frequencies in
    [f_lo, f_hi] cycles per unit, random directions and phases, amplitude
    proportional to 1/f, scaled to the given standard deviation."""
    f = np.exp(rng.uniform(math.log(f_lo), math.log(f_hi), size=(n_waves, 3)))
    th = rng.uniform(0, 2 * math.pi, size=(n_waves, 3))
    k = 2 * math.pi * f[:, None, :] * np.stack([np.cos(th), np.sin(th)], axis=1)  # (n, 2, 3)
    ph = rng.uniform(0, 2 * math.pi, size=(n_waves, 3))
    amp = 1.0 / f
    amp *= std / np.sqrt(0.5 * (amp ** 2).sum(axis=0, keepdims=True))

    def tex(uv):
        out = np.zeros((uv.shape[0], 3))
        for w in range(n_waves):
            for ch in range(3):
                out[:, ch] += amp[w, ch] * np.sin(uv @ k[w, :, ch] + ph[w, ch])
        return out
    return tex


def textured_scene(n: int, seed: int, n_surfaces: int = 400, size_range=(0.04, 0.9), shell_radius: float = 12.0,
                   cover: float = 1.0, log_scale_std: float = 0.3, tex_f_hi: float = 40.0, tex_waves: int = 32,
                   dtype=np.float32) -> np.ndarray:
    """(n, 59) Gaussians on textured planes/spheres plus a background shell.

    Layout: a dead-leaves arrangement, the classic model of natural-image
    statistics -- ``n_surfaces`` plane patches and spheres with half-sizes drawn
    from the scale-invariant density p(s) ~ s^-3 on ``size_range`` (equal
    surface area per octave of size), placed at random in [-1.8, 1.8]^3, each
    with its own base colour and a 1/f texture, so views have edges and
    texture at every scale.  Gaussians are spread over the surfaces in
    proportion to area (10% on the shell).  Scales follow the local density:
    the mean scale is ``cover`` times the mean spacing sqrt(area / count), with
    a log-normal spread, so surfaces are closed and resolved down to the
    Gaussian spacing."""
    rng = np.random.default_rng(seed)
    g = np.zeros((n, NPARAM), dtype=dtype)
    n_shell = n // 10
    n_surf = n - n_shell
    lo, hi = size_range
    # inverse CDF of p(s) ~ s^-3 on [lo, hi]
    u = rng.uniform(size=n_surfaces)
    size = 1.0 / np.sqrt(1.0 / lo ** 2 - u * (1.0 / lo ** 2 - 1.0 / hi ** 2))
    is_plane = np.arange(n_surfaces) % 2 == 0
    area = np.where(is_plane, (2.0 * size) ** 2, 4.0 * math.pi * size ** 2)
    counts = np.floor(n_surf * area / area.sum()).astype(np.int64)
    counts[np.argsort(-area)[: n_surf - counts.sum()]] += 1
    means = np.zeros((n, 3))
    dc = np.zeros((n, 3))
    log_sigma = np.zeros(n)
    o = 0
    for s in range(n_surfaces):
        m = int(counts[s])
        centre = rng.uniform(-1.8, 1.8, size=3)
        tex = _band_noise(rng, n_waves=tex_waves, f_hi=tex_f_hi)
        base = rng.uniform(0.1, 0.9, size=3)
        if m == 0:
            continue
        uv = rng.uniform(-1.0, 1.0, size=(m, 2))
        if is_plane[s]:
            a = rng.normal(size=3); a /= np.linalg.norm(a)
            b = np.cross(a, rng.normal(size=3)); b /= np.linalg.norm(b)
            means[o:o + m] = centre + size[s] * (uv[:, :1] * a + uv[:, 1:] * b)
        else:
            th = np.arccos(uv[:, 0])
            ph = math.pi * uv[:, 1]
            d = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
            means[o:o + m] = centre + size[s] * d
        log_sigma[o:o + m] = math.log(cover * math.sqrt(area[s] / m))
        dc[o:o + m] = base + tex(uv * size[s] / 0.65)  # texture frequency in world units
        o += m
    d = rng.normal(size=(n_shell, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    means[o:] = shell_radius * d
    log_sigma[o:] = math.log(cover * math.sqrt(4.0 * math.pi * shell_radius ** 2 / max(n_shell, 1)))
    sky = _band_noise(rng, f_hi=20.0)
    dc[o:] = 0.5 + sky(d[:, :2] * 4.0)
    g[:, 0:3] = means
    g[:, 3:6] = log_sigma[:, None] + rng.normal(0.0, log_scale_std, size=(n, 3))
    q = rng.normal(size=(n, 4))
    g[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True)
    g[:, 10] = rng.normal(0.0, 1.0, size=n)
    g[:, 11:59] = rng.normal(0.0, 0.2, size=(n, 48))
    g[:, 11:14] = (np.clip(dc, 0.0, 1.0) - 0.5) / SH_DC_NORM
    return g


def perturb(g: np.ndarray, seed: int, mean_sigma: float = 0.01, n_keep: int | None = None,
            dtype=np.float32) -> np.ndarray:
    """Initial state for optimisation: a subset of ``g`` with jittered means,
    isotropic scales, opacity 0.1 and higher-order SH set to zero."""
    rng = np.random.default_rng(seed)
    idx = np.arange(g.shape[0]) if n_keep is None else np.sort(rng.choice(g.shape[0], n_keep, replace=False))
    out = np.array(g[idx], dtype=dtype)
    out[:, 0:3] += rng.normal(0.0, mean_sigma, size=(len(idx), 3))
    out[:, 3:6] = out[:, 3:6].mean(axis=1, keepdims=True)
    out[:, 6:10] = np.array([1.0, 0.0, 0.0, 0.0])
    out[:, 10] = math.log(0.1 / 0.9)
    out[:, 14:59] = 0.0
    return out


def jitter(g: np.ndarray, seed: int, mean_sigma: float = 0.01, scale_sigma: float = 0.1,
           opacity_sigma: float = 0.2, sh_sigma: float = 0.05, dtype=np.float32) -> np.ndarray:
    """A nearby optimisation state: ``g`` with Gaussian noise on every parameter."""
    rng = np.random.default_rng(seed)
    out = np.array(g, dtype=dtype)
    n = out.shape[0]
    out[:, 0:3] += rng.normal(0.0, mean_sigma, size=(n, 3)).astype(dtype)
    out[:, 3:6] += rng.normal(0.0, scale_sigma, size=(n, 3)).astype(dtype)
    out[:, 6:10] += rng.normal(0.0, 0.05, size=(n, 4)).astype(dtype)
    out[:, 10] += rng.normal(0.0, opacity_sigma, size=n).astype(dtype)
    out[:, 11:59] += rng.normal(0.0, sh_sigma, size=(n, 48)).astype(dtype)
    return out
