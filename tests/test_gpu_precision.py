"""Mixed-precision records (float16 conic/opacity, bfloat16 colour) against
the FP64 oracle (needs a GPU).

Two checks.  (1) Kernel correctness: the oracle fed the DEQUANTIZED records
(the exact values the kernels widen to float32) must match the mixed path to
the float32 tolerances of the full-precision path.  (2) Precision error: the
oracle fed the float32 master records measures what the storage format costs.
Derived bound for (2): float16 keeps 11 significant bits (relative rounding
<= 2^-11 = 4.9e-4), bfloat16 8 (<= 2^-8 = 3.9e-3).  The exponent of alpha is
at most 2 ln 255 / 2 = 5.5 in magnitude, so its relative error stays below
5.5 * 4.9e-4 = 2.7e-3; colour below 3.9e-3; a Gaussian whose alpha crosses
1/255 because of rounding adds or removes at most (1/255) * T * c <= 4e-3.
A pixel blends a few dozen Gaussians with weights summing to <= 1, so its
error is bounded by about 2e-2 and is typically two orders smaller: the test
asserts max <= 2e-2 and mean <= 1e-3, and prints the measured values.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2503_18402_gb300 import capi, synth  # noqa: E402
from paper_2503_18402_gb300.raster import Rasterizer  # noqa: E402
from tests import _gpu as G  # noqa: E402

pytestmark = pytest.mark.gpu


def _bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _decode(packed, n):
    raw = G.np_(packed[: n * 24]).reshape(n, 24)
    uv = raw[:, 0:8].copy().view(np.float32).reshape(n, 2)
    h = raw[:, 8:16].copy().view(np.float16).reshape(n, 4)
    bf = raw[:, 16:22].copy().view(np.uint16).reshape(n, 3).astype(np.uint32) << 16
    col = bf.view(np.float32)
    return np.concatenate([uv, h.astype(np.float32), col], axis=1).astype(np.float64)  # u v A B C o r g b


def _setup(W, H, n, seed, tile):
    g = synth.random_gaussians(n, seed)
    g[:, 3:6] += 0.3
    cam = synth.camera_cfg0(W, H, 4.0)
    bg = (0.2, 0.1, 0.3)
    out = {}
    for rec in (0, 1):
        rz = Rasterizer("cuda", capi.raster_opts(tile=tile, bg=bg, record=rec))
        params = G.gpu_params(g)
        fr = rz.forward(params, n, G.gpu_camera(cam), examined=True)
        rng = np.random.default_rng(seed)
        dL = (rng.normal(size=(3, H, W)) / (3 * H * W)).astype(np.float32)
        rz.backward(params, fr, torch.from_numpy(dL).cuda(), torch.empty_like(params))
        torch.cuda.synchronize()
        out[rec] = (rz, fr, dL)
    return g, cam, bg, out


def test_packing_rounds_to_nearest():
    g, cam, bg, out = _setup(64, 64, 2000, 3, 16)
    rz, fr, _ = out[1]
    n = g.shape[0]
    f32 = G.np_(rz.feat[:n]).astype(np.float64)
    dec = _decode(rz.packed, n)
    vis = G.np_(rz.radius[:n]) > 0
    np.testing.assert_array_equal(dec[vis, 0:2], f32[vis, 0:2])
    np.testing.assert_array_equal(dec[vis, 2:6], f32[vis, 2:6].astype(np.float16).astype(np.float64))
    np.testing.assert_array_equal(dec[vis, 6:9], _bf16_round(f32[vis, 6:9]))


@pytest.mark.parametrize("W,H,tile", [(64, 64, 16), (130, 99, 8)])
def test_mixed_records_kernel_matches_oracle_on_dequantized_records(W, H, tile):
    g, cam, bg, out = _setup(W, H, 5000, 7 + W, tile)
    rz, fr, dL = out[1]
    n = g.shape[0]
    dec = _decode(rz.packed, n)
    gid = G.np_(rz.gid[: fr.M]).view(np.uint32)
    ranges = G.np_(rz.ranges[: rz.n_tiles]).view(np.uint32)
    k = oracle.consts(tile=tile)
    orf = oracle.render_fwd(dec, W, H, tile, gid, ranges, G.f32(bg), k)
    assert np.abs(G.np_(fr.img) - orf["img"]).max() <= 1e-5
    np.testing.assert_array_equal(G.np_(fr.last), orf["last"])
    og2 = oracle.render_bwd(dec, W, H, tile, gid, ranges, G.f32(bg), k, dL.astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(rz.grad2d[:n])[:, :9], og2)
    assert ok, (worst, nbad)


def test_mixed_precision_error_against_float32_master_records():
    W, H, tile = 64, 64, 16
    g, cam, bg, out = _setup(W, H, 6000, 11, tile)
    rz, fr, dL = out[1]
    n = g.shape[0]
    f32 = G.np_(rz.feat[:n]).astype(np.float64)[:, :9]
    gid = G.np_(rz.gid[: fr.M]).view(np.uint32)
    ranges = G.np_(rz.ranges[: rz.n_tiles]).view(np.uint32)
    k = oracle.consts(tile=tile)
    orf = oracle.render_fwd(f32, W, H, tile, gid, ranges, G.f32(bg), k)
    err = np.abs(G.np_(fr.img) - orf["img"])
    og2 = oracle.render_bwd(f32, W, H, tile, gid, ranges, G.f32(bg), k, dL.astype(np.float64))
    g2 = G.np_(rz.grad2d[:n])[:, :9]
    rel = np.linalg.norm(g2 - og2) / max(np.linalg.norm(og2), 1e-30)
    print(f"mixed-precision records, 64x64: image max {err.max():.3e} mean {err.mean():.3e}; "
          f"2D gradient relative L2 {rel:.3e}")
    assert err.max() <= 2e-2 and err.mean() <= 1e-3
    assert rel <= 5e-2


def test_mixed_precision_error_at_full_scale_crop():
    """The reduced-precision workload: a 6M-Gaussian scene, one 1600x1063
    view, mixed records; error against the FP64 oracle (fed the float32
    master records and the same pair lists) on a centred 64x64 crop, for the
    image and for the 2D gradients of a loss supported on the crop."""
    W, H, tile = 1600, 1063, 8
    gt = synth.textured_scene(6_000_000, 1004)
    cams = synth.ring_cameras(300, W, H, 5.0, 2004)
    v = cams[17]
    cam = G.gpu_camera(v)
    params = G.gpu_params(gt)
    n = gt.shape[0]
    rz = Rasterizer("cuda", capi.raster_opts(tile=tile, record=1))
    fr = rz.forward(params, n, cam)
    x0, y0 = (W - 64) // 2 // tile * tile, (H - 64) // 2 // tile * tile
    rng = np.random.default_rng(5)
    dL = np.zeros((3, H, W), np.float32)
    dL[:, y0:y0 + 64, x0:x0 + 64] = rng.normal(size=(3, 64, 64)) / (3 * 64 * 64)
    rz.backward(params, fr, torch.from_numpy(dL).cuda(), torch.empty_like(params))
    torch.cuda.synchronize()
    f32 = G.np_(rz.feat[:n]).astype(np.float64)[:, :9]
    gid = G.np_(rz.gid[: fr.M]).view(np.uint32)
    ranges = G.np_(rz.ranges[: rz.n_tiles]).view(np.uint32)
    k = oracle.consts(tile=tile)
    py, px = np.mgrid[y0:y0 + 64, x0:x0 + 64]
    o = oracle.render_pixels(f32, W, tile, gid, ranges, np.zeros(3), k, px.ravel(), py.ravel())
    got = G.np_(fr.img)[:, y0:y0 + 64, x0:x0 + 64].reshape(3, -1).T
    err = np.abs(got - o["rgb"])
    og2 = oracle.render_bwd(f32, W, H, tile, gid, ranges, np.zeros(3), k, dL.astype(np.float64))
    g2 = G.np_(rz.grad2d[:n])[:, :9]
    touched = np.abs(og2).sum(axis=1) > 0
    rel = np.linalg.norm(g2[touched] - og2[touched]) / max(np.linalg.norm(og2[touched]), 1e-30)
    print(f"mixed-precision records, 6M Gaussians, 1600x1063, 64x64 crop: image max {err.max():.3e} "
          f"mean {err.mean():.3e}; 2D gradient relative L2 {rel:.3e} over {int(touched.sum())} Gaussians")
    assert err.max() <= 2e-2 and err.mean() <= 1e-3
    assert rel <= 5e-2
