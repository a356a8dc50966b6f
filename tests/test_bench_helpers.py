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
