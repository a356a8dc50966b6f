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
