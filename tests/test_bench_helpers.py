"""Host logic of bench.py that needs no GPU: launch-shape labels and the
roofline's traffic field, which is read from a committed ncu summary only
while the kernel's source file is the one the summary was taken on."""
from __future__ import annotations

import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_shape_labels_round_trip():
    from paper_2503_18402_gb300.autotune import CANDIDATES
    for s in CANDIDATES:
        assert bench.parse_shape(s.label()) == s
    with pytest.raises(SystemExit):
        bench.parse_shape("t8f1b1")


def _tree(tmp_path, source: bytes, profile_sha: str, stage="render_bwd", nbytes=123456):
    src = tmp_path / "paper_2503_18402_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "render.cu").write_bytes(source)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text(f"# summary\n\n    ncu ... (command)\n\nstage: {stage}\nsource_sha1: {profile_sha}\n"
                               f"dram_bytes_per_launch: {nbytes}\n\n| a | b |\n")
    return str(tmp_path)


def test_traffic_read_when_the_source_matches(tmp_path):
    code = b"__global__ void k() {}\n"
    root = _tree(tmp_path, code, hashlib.sha1(code).hexdigest())
    assert bench.measured_traffic("render_bwd", root) == 123456
    assert bench.measured_traffic("render_fwd", root) is None  # no summary for that stage


def test_traffic_null_once_the_kernel_changed(tmp_path):
    root = _tree(tmp_path, b"__global__ void k() { /* edited */ }\n", hashlib.sha1(b"old").hexdigest())
    assert bench.measured_traffic("render_bwd", root) is None
    assert bench.measured_traffic("no_such_stage", root) is None


def test_banded_oracle_step_equals_the_whole_view_oracle():
    """The CPU baseline splits one oracle step over host threads (Gaussian
    chunks, tile-row bands with a halo for SSIM); its image, loss gradient,
    2D gradients and parameter gradients equal the whole-view oracle's."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import oracle
    from oracle import ssim as ossim
    from paper_2503_18402_gb300 import synth
    W, H, B = 96, 70, 8
    g = np.asarray(synth.random_gaussians(1500, 21), np.float64)
    cam = synth.camera_cfg0(W, H, 3.5)
    tgt = synth.target_image(W, H, 22)
    with ThreadPoolExecutor(3) as pool:
        _, info = bench.oracle_step(g, cam, W, H, B, tgt, pool, 3, keep=True)
    assert info["bands"] > 3 and info["chunks"] == 3
    fx, fy, cx, cy = cam["intr"]
    ocam = oracle.camera(cam["viewmat"], fx, fy, cx, cy, W, H)
    k = oracle.consts(tile=B)
    f = oracle.forward(g, ocam, k)
    np.testing.assert_allclose(info["img"], f["img"], rtol=0, atol=1e-12)
    loss, dL = ossim.l1_dssim(f["img"], tgt)
    assert info["loss"] == pytest.approx(loss, rel=1e-12)
    np.testing.assert_allclose(info["dL"], dL, rtol=0, atol=1e-15)
    ob = oracle.backward(g, ocam, k, f, dL)
    np.testing.assert_allclose(info["grad2d"], ob["grad2d"], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(info["grad"], ob["grad"], rtol=1e-9, atol=1e-13)
