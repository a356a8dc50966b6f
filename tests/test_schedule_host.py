"""The library's host-side schedule (dg_schedule_*) against the FP64 schedule
oracle (Sec. 4.2-4.3, Eq. 4/5/7).  CPU only: these calls do no device work;
the summed-area table they consume is built here with numpy from the oracle's
spectrum (the GPU path that produces it is checked in tests/test_gpu_schedule.py)."""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import schedule as sch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2503_18402_gb300 import build
    build.build()
    from paper_2503_18402_gb300 import capi as c
    return c


def _sat(Mbar):
    H, W = Mbar.shape
    s = np.zeros((H + 1, W + 1))
    s[1:, 1:] = Mbar.cumsum(0).cumsum(1)
    return s


def _images(kind, H, W, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "cosine":
        x = np.arange(W)
        row = 0.5 + 0.3 * np.cos(2 * math.pi * 6 * x / W)
        img = np.broadcast_to(row[None, :], (H, W))
        return np.stack([img] * 3)[None]
    ky = np.fft.fftfreq(H)[:, None]; kx = np.fft.fftfreq(W)[None, :]
    amp = 1 / np.maximum(np.hypot(ky, kx), 1 / max(H, W)) ** 1.1
    imgs = np.stack([[np.real(np.fft.ifft2(amp * np.exp(2j * math.pi * rng.uniform(size=(H, W)))))
                      for _ in range(3)] for _ in range(3)])
    return imgs - imgs.min() + 0.05


def test_struct_layouts_match_the_header(capi):
    src = os.path.join(ROOT, "_build_layout_probe.c")
    exe = os.path.join(ROOT, "_build_layout_probe")
    code = ('#include <stdio.h>\n#include <stddef.h>\n#include "include/dashgs.h"\n'
            'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(dg_sched_params), sizeof(dg_schedule),'
            ' sizeof(dg_sched_out), offsetof(dg_schedule, k_full), offsetof(dg_schedule, s), sizeof(dg_camera),'
            ' sizeof(dg_raster_opts)); return 0;}\n')
    try:
        with open(src, "w") as f:
            f.write(code)
        subprocess.check_call(["gcc", "-I", ROOT, "-o", exe, src])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    finally:
        for p in (src, exe):
            if os.path.exists(p):
                os.remove(p)
    want = [ctypes.sizeof(capi.SchedParams), ctypes.sizeof(capi.Schedule), ctypes.sizeof(capi.SchedOut),
            capi.Schedule.k_full.offset, capi.Schedule.s.offset, ctypes.sizeof(capi.Camera),
            ctypes.sizeof(capi.RasterOpts)]
    assert got == want


@pytest.mark.parametrize("kind,H,W,S", [("cosine", 32, 48, 30000), ("pink", 48, 64, 3000), ("pink", 41, 57, 5000)])
def test_host_schedule_matches_oracle(capi, kind, H, W, S):
    Mb = sch.spectrum_mean(_images(kind, H, W))
    ref = sch.ResolutionSchedule(Mb, S, a=4.0)
    p = capi.sched_params(S, a=4.0, P_init=1e5, P_cap=0.0, lr_pos_init=1.6e-4, lr_pos_final=1.6e-6)
    s = capi.dg_schedule_init(_sat(Mb), H, W, p)
    assert s.m == ref.m
    assert s.X0 == pytest.approx(ref.X0, rel=1e-12)
    assert s.r_m == pytest.approx(ref.r_m, rel=1e-10)
    for i in range(ref.m + 1):
        assert s.X[i] == pytest.approx(ref.X[i], rel=1e-12)
        assert s.r[i] == pytest.approx(ref.r[i], rel=1e-10)
        assert s.s[i] == pytest.approx(ref.s[i], rel=1e-10, abs=1e-7)
    k_full = ref.first_full_res_iter()
    assert s.k_full == k_full
    for k in range(0, S + 1, max(1, S // 997)):
        o = capi.dg_schedule_step(s, k)
        assert o.r_mod == ref.r_mod(k)
        assert o.r_cont == pytest.approx(ref.r_cont(k), rel=1e-10)
        assert (o.height, o.width) == ref.render_size(k)
        assert o.lr_pos == pytest.approx(sch.position_lr(k, k_full, S, 1.6e-4, 1.6e-6), rel=1e-12)
        assert o.P_target == pytest.approx(sch.primitive_target(k, S, ref.r_mod(k), 1e5, 5e5), rel=1e-12)


def test_host_primitive_budget_eq5(capi):
    Mb = sch.spectrum_mean(_images("pink", 48, 64))
    S = 30000
    s = capi.dg_schedule_init(_sat(Mb), 48, 64, capi.sched_params(S, P_init=1e5, P_cap=3e6))
    P_fin = 5e5
    rs = sch.ResolutionSchedule(Mb, S)
    rng = np.random.default_rng(0)
    for k in range(500, 15001, 100):
        P_add = int(rng.integers(0, 40000))
        o = capi.dg_schedule_densify(s, k, P_add)
        P_fin = sch.pfin_update(P_fin, P_add)
        assert s.P_fin == pytest.approx(P_fin, rel=1e-12)
        want = min(3e6, sch.primitive_target(k, S, rs.r_mod(k), 1e5, P_fin))
        assert o.P_target == pytest.approx(want, rel=1e-12)


def test_plain_schedule_full_resolution_and_backbone_lr(capi):
    S, H, W = 30000, 822, 1237
    p = capi.sched_params(S, P_init=1e5, lr_pos_init=1.6e-4 * 5, lr_pos_final=1.6e-6 * 5)
    s = capi.dg_schedule_init_plain(H, W, p)
    assert s.k_full == 0 and s.m == 0
    for k in list(range(0, S + 1, 997)) + [S, S + 50]:
        o = capi.dg_schedule_step(s, k)
        assert (o.r_mod, o.height, o.width) == (1, H, W)
        assert o.lr_pos == pytest.approx(sch.position_lr(k, 0, S, 8e-4, 8e-6), rel=1e-12)
    # the backbone's exponential decay: halfway, the geometric mean of the two ends
    assert capi.dg_schedule_step(s, S // 2).lr_pos == pytest.approx(math.sqrt(8e-4 * 8e-6), rel=1e-12)


def test_densify_budget_eq4_eq5_and_cap(capi):
    Mb = sch.spectrum_mean(_images("pink", 48, 64))
    S = 30000
    P_init, P_cap = 1e5, 1.2e6
    s = capi.dg_schedule_init(_sat(Mb), 48, 64, capi.sched_params(S, P_init=P_init, P_cap=0.0))
    rs = sch.ResolutionSchedule(Mb, S)
    rng = np.random.default_rng(3)
    P_fin = 5 * P_init
    n_keep = int(P_init)
    for k in range(500, 15001, 100):
        n_cand = int(rng.integers(0, 60000))
        b, o = capi.dg_densify_budget(s, k, n_keep, n_cand, int(P_cap))
        P_fin = sch.pfin_update(P_fin, n_cand)
        target = sch.primitive_target(k, S, rs.r_mod(k), P_init, P_fin)
        assert o.P_target == pytest.approx(target, rel=1e-12)
        want = max(0, min(math.floor(target) - n_keep, int(P_cap) - n_keep))
        assert b == want
        n_keep = n_keep + min(b, n_cand) - int(rng.integers(0, 2000))
    # the backbone (no schedule): every candidate, up to the cap
    assert capi.dg_densify_budget(None, 100, 1000, 500, 0)[0] == 500
    assert capi.dg_densify_budget(None, 100, 1000, 500, 1200)[0] == 200
    assert capi.dg_densify_budget(None, 100, 1300, 500, 1200)[0] == 0


def test_camera_scale_moves_pixels_with_the_image(capi):
    """A point's pixel coordinate in a w x h render of the same view is its
    full-resolution coordinate times w/W (and h/H): the render covers the same
    field of view with fewer pixels."""
    rng = np.random.default_rng(0)
    vm = np.concatenate([np.eye(3), [[0.1], [-0.2], [4.0]]], axis=1)
    full = capi.camera(vm.reshape(-1), 1071.2, 1071.2, 618.5, 411.0, 1237, 822)
    X = rng.uniform(-1, 1, size=(50, 3))

    def pix(c):
        v = np.array(c.viewmat[:], dtype=np.float64).reshape(3, 4)
        x = X @ v[:, :3].T + v[:, 3]
        return np.stack([c.fx * x[:, 0] / x[:, 2] + c.cx, c.fy * x[:, 1] / x[:, 2] + c.cy], 1)

    for w, h in ((309, 205), (618, 411), (95, 63), (1237, 822)):
        c = capi.dg_camera_scale(full, w, h)
        assert (c.width, c.height) == (w, h)
        assert list(c.viewmat) == list(full.viewmat)
        np.testing.assert_allclose(pix(c), pix(full) * [w / 1237, h / 822], rtol=1e-6, atol=1e-4)
    with pytest.raises(capi.DashGSError):
        capi.dg_camera_scale(full, 0, 10)


def test_batch_adam_scale(capi):
    lr = [0.1 * (i + 1) for i in range(59)]
    same, b1, b2 = capi.dg_batch_adam_scale(1, lr, 0.9, 0.999)
    assert same == pytest.approx(lr, rel=1e-7) and (b1, b2) == pytest.approx((0.9, 0.999), rel=1e-7)
    out, b1, b2 = capi.dg_batch_adam_scale(16, lr, 0.9, 0.999)
    assert out == pytest.approx([4 * x for x in lr], rel=1e-7)
    assert b1 == pytest.approx(0.9 ** 16, rel=1e-6) and b2 == pytest.approx(0.999 ** 16, rel=1e-6)
    with pytest.raises(capi.DashGSError):
        capi.dg_batch_adam_scale(0, lr, 0.9, 0.999)
