"""The C-ABI library builds, loads and exports every entry point that
include/dashgs.h declares (CPU only: no compute call reaches the GPU)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dashgs.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^DG_API\s+[\w\s\*]+?\b(dg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_18402_gb300 import build
    path = build.build()
    return path, ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dg_project", "dg_bin_count", "dg_bin_sort", "dg_render_fwd", "dg_render_bwd",
                     "dg_project_bwd", "dg_loss_l1", "dg_adam_step"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    path, L = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dg_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(L, n)
    # nothing else leaks out of the library under a dg_ name
    assert exported <= set(_declared())


def test_binding_covers_every_export():
    from paper_2503_18402_gb300 import capi
    assert set(capi.EXPORTS) == set(_declared())


def test_host_only_calls_without_gpu():
    from paper_2503_18402_gb300 import capi
    assert capi.dg_abi_version() == 7
    assert capi.dg_bin_workspace_size(1000, 1, 5000) > 5000 * 16
    assert capi.dg_bin_workspace_size(1000, 4, 5000) > capi.dg_bin_workspace_size(1000, 1, 5000)
    assert capi.dg_bin_workspace_size(-1, 1, 0) == 0
    assert capi.dg_bin_workspace_size(10, 17, 0) == 0  # more views than one call takes
    cam1 = capi.camera([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 4], 50, 50, 32, 32, 64, 64)
    nosplit = capi.dg_render_workspace_size(cam1, 1, capi.raster_opts(split_len=-1))
    split = capi.dg_render_workspace_size(cam1, 1, capi.raster_opts())
    assert nosplit >= 16 and split > nosplit
    # one flag byte per pair on top of the fixed part
    assert capi.dg_render_workspace_size(cam1, 1, capi.raster_opts(), 1 << 20) == split + (1 << 20)
    big = capi.camera([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 4], 50, 50, 32, 32, 1600, 1063)
    assert capi.dg_render_workspace_size([big] * 16, 16, capi.raster_opts(tile=8)) > \
        capi.dg_render_workspace_size(big, 1, capi.raster_opts(tile=8))
    assert capi.dg_render_workspace_size(cam1, 1, capi.raster_opts(tile=12)) == 0
    assert capi.dg_loss_workspace_size(100) >= 4
    # argument validation happens on the host before any launch
    opts = capi.raster_opts(sh_degree=7)
    cam = capi.camera([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 4], 50, 50, 32, 32, 64, 64)
    with pytest.raises(capi.DashGSError) as e:
        capi.dg_project(1 << 20, 8, 8, cam, 1, opts, 1 << 21, 1 << 22, 1 << 23, 1 << 24, 1 << 25)
    assert e.value.status == capi.DG_ERR_ARG and "sh_degree" in capi.dg_last_error()
    with pytest.raises(capi.DashGSError) as e:
        capi.dg_render_fwd(1 << 20, 1 << 21, 1 << 22, cam, 1, capi.raster_opts(tile=12), 1, 2, 3, None, None,
                           1 << 26, 256)
    assert "tile" in str(e.value)
    with pytest.raises(capi.DashGSError) as e:
        capi.dg_project(1 << 20, 8, 8, [cam] * 17, 17, capi.raster_opts(), 1 << 21, 1 << 22, 1 << 23, 1 << 24,
                        1 << 25)
    assert "n_views" in str(e.value)
