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
