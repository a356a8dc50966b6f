"""Helpers for GPU parity tests: move seeded inputs to both sides.

The CUDA path takes float32 planar [59, P] parameters; the oracle takes the
same float32 values widened to float64, (P, 59).  The projected record of the
CUDA path is (u, v, A, B | C, o, r, g | b, 0, 0, 0); its first nine floats are
the oracle's feature record (u, v, A, B, C, o, r, g, b), and likewise for the
2D gradients.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2503_18402_gb300 import capi

DEV = "cuda"


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def gpu_params(g: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(np.asarray(g, np.float32).T)).to(DEV)


def gpu_camera(cam: dict) -> capi.Camera:
    fx, fy, cx, cy = cam["intr"]
    return capi.camera(np.asarray(cam["viewmat"], np.float32).reshape(-1), fx, fy, cx, cy,
                       cam["width"], cam["height"])


def oracle_camera(cam: dict) -> oracle.Camera:
    fx, fy, cx, cy = (float(np.float32(v)) for v in cam["intr"])
    return oracle.camera(f32(cam["viewmat"]), fx, fy, cx, cy, cam["width"], cam["height"])


def np_(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def grad_close(gpu, ref, rtol=1e-4, atol=1e-6):
    """Gradient tolerance: 1e-4 relative, 1e-6 absolute near zero."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref)
    bad = err > rtol * np.abs(ref) + atol
    return (not bad.any()), float((err / (np.abs(ref) + atol)).max(initial=0.0)), int(bad.sum())
