"""Finite-difference pins of the oracle's analytic backward (Sec. 3: the
rasterizer is differentiated end to end).

Central differences in FP64, h = 1e-6 max(1, |theta|), on tiny scenes.  A
parameter is only compared when the discrete structure (radius, tile lists,
last contributor, examined count of every pixel) is identical at theta +/- h,
i.e. the scene has a margin at every threshold for that perturbation.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2503_18402_gb300 import synth
from tests import _util as U


def _loss_and_struct(g, cam, k, wts, bg):
    out = oracle.forward(g, cam, k, bg=bg)
    L = float(np.sum(wts * out["img"]))
    struct = (out["proj"]["radius"].tobytes(), out["bins"]["gid"].tobytes(),
              out["last"].tobytes(), out["examined"].tobytes(),
              out["proj"]["clamp"].tobytes())
    return L, struct, out


def _fd_check(g, camd, k, bg=(0.0, 0.0, 0.0), seed=0, min_frac=0.9):
    cam = U.oracle_cam(oracle, camd)
    rng = np.random.default_rng(seed)
    W, H = camd["width"], camd["height"]
    wts = rng.normal(size=(3, H, W))
    L0, s0, out = _loss_and_struct(g, cam, k, wts, bg)
    an = oracle.backward(g, cam, k, out, wts, bg=bg)["grad"]
    n_sh = (k.sh_degree + 1) ** 2
    active = list(range(11 + 3 * n_sh))
    scale = np.abs(an).max()
    checked = skipped = 0
    worst = 0.0
    for i in range(g.shape[0]):
        for j in active:
            h = 1e-6 * max(1.0, abs(g[i, j]))
            gp = g.copy(); gp[i, j] += h
            gm = g.copy(); gm[i, j] -= h
            Lp, sp, _ = _loss_and_struct(gp, cam, k, wts, bg)
            Lm, sm, _ = _loss_and_struct(gm, cam, k, wts, bg)
            if sp != s0 or sm != s0:
                skipped += 1
                continue
            fd = (Lp - Lm) / (2 * h)
            err = abs(fd - an[i, j])
            tol = 1e-6 * abs(an[i, j]) + 1e-8 * scale
            worst = max(worst, err / (abs(an[i, j]) + 1e-12))
            assert err <= tol, (i, j, fd, an[i, j])
            checked += 1
    assert checked >= min_frac * (checked + skipped), (checked, skipped)
    # parameters beyond the SH degree carry no gradient
    assert np.all(an[:, 11 + 3 * n_sh:] == 0)
    return checked


def _tiny_scene(n, seed, W=32, H=32, f=30.0):
    rng = np.random.default_rng(seed)
    g = synth.random_gaussians(n, seed)
    g[:, 0:2] = rng.uniform(-0.6, 0.6, size=(n, 2))
    g[:, 2] = rng.uniform(2.0, 3.5, size=n)
    g[:, 3:6] = rng.normal(-1.8, 0.3, size=(n, 3))
    g[:, 6:10] = rng.normal(size=(n, 4))  # unnormalised: exercises the normalisation adjoint
    return g, U.identity_cam(W, H, f)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fd_random_tiny_scene(seed):
    g, cam = _tiny_scene(6, seed)
    _fd_check(g, cam, oracle.consts(sh_degree=3), seed=seed)


def test_fd_with_background_and_low_sh_degree():
    g, cam = _tiny_scene(5, 7)
    _fd_check(g, cam, oracle.consts(sh_degree=1), bg=(0.3, 0.6, 0.2), seed=7)


def test_fd_rotated_camera_and_clamped_colour():
    g = synth.random_gaussians(5, 9)
    g[:, 3:6] = -1.5
    g[:, 11:59] *= 4.0  # some colour channels clamp at 0
    cam = synth.camera_cfg0(32, 32, 4.0)
    cam["intr"] = (30.0, 30.0, 16.0, 16.0)
    k = oracle.consts(sh_degree=3)
    pr = oracle.project(g, U.oracle_cam(oracle, cam), k)
    assert pr["clamp"][pr["radius"] > 0].any()
    _fd_check(g, cam, k, seed=9)


def test_fd_frustum_guard_and_alpha_clamp():
    # Gaussian 0: centre beyond the guarded frustum, footprint reaches the image
    # Gaussian 1: nearly opaque, alpha clamps at 0.99 near its centre
    g0 = U.single_gaussian((1.7, 0.2, 2.0), [math.log(0.7), math.log(0.5), math.log(0.4)],
                           quat=(0.9, 0.2, -0.3, 0.1), opacity=0.8, dc=(0.6, 0.4, 0.7))
    g1 = U.single_gaussian((-0.1, 0.15, 2.6), [math.log(0.25), math.log(0.2), math.log(0.3)],
                           quat=(0.7, -0.1, 0.4, 0.2), opacity=0.9995, dc=(0.2, 0.9, 0.4))
    rng = np.random.default_rng(4)
    g = np.concatenate([g0, g1])
    g[:, 14:59] = rng.normal(0, 0.2, size=(2, 45))
    cam = U.identity_cam(32, 32, 30.0)
    k = oracle.consts(sh_degree=3)
    pr = oracle.project(g, U.oracle_cam(oracle, cam), k)
    assert pr["radius"][0] > 0 and 1.7 / 2.0 > 1.3 * 16 / 30.0
    _fd_check(g, cam, k, seed=4)


def test_fd_deep_stack_division_path():
    # many coincident-ish footprints: exercises the suffix-colour adjoint
    rng = np.random.default_rng(8)
    rows = []
    for i in range(8):
        z = 2.0 + 0.15 * i
        rows.append(U.single_gaussian((rng.normal(0, 0.05), rng.normal(0, 0.05), z),
                                      np.log([0.15 * z / 2, 0.12 * z / 2, 0.1]),
                                      quat=tuple(rng.normal(size=4)), opacity=rng.uniform(0.3, 0.8),
                                      dc=tuple(rng.uniform(0.1, 0.9, 3))))
    g = np.concatenate(rows)
    _fd_check(g, U.identity_cam(32, 32, 30.0), oracle.consts(sh_degree=0), bg=(0.5, 0.5, 0.5), seed=8)


@pytest.mark.parametrize("seed", [4, 5])
def test_fd_mip_2d_filter(seed):
    """Mip-Splatting's 2D filter (backbone variant): the opacity compensation
    sqrt(det(S2) / det(S2 + s I)) is differentiated through the covariance;
    smaller Gaussians (log-scale -3.2) so that the compensation is far from 1."""
    g, cam = _tiny_scene(6, seed)
    g[:, 3:6] = np.random.default_rng(seed).normal(-3.2, 0.3, size=(6, 3))
    _fd_check(g, cam, oracle.consts(sh_degree=1, mip2d=0.1), seed=seed)
