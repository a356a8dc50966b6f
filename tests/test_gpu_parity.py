"""CUDA path vs the FP64 oracle, element by element (needs a GPU).

Tolerances (from the target: tile lists and key order bit-exact; images
within 1e-5 absolute; gradients within 1e-4 relative or 1e-6 absolute near
zero).  Intermediate projected records are FP32 results of an FP64
definition; their tolerances follow from the FP32 arithmetic (a few ulps of
the pixel coordinates, 1e-4 relative on the conic whose 2x2 inverse has
condition number up to ~10 on these scenes).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2503_18402_gb300 import capi, synth  # noqa: E402
from paper_2503_18402_gb300.raster import Rasterizer, rasterize  # noqa: E402
from tests import _gpu as G  # noqa: E402
from tests import _util as U  # noqa: E402

pytestmark = pytest.mark.gpu


def _setup(g, cam, bg=(0.0, 0.0, 0.0), tile=16, sh=3):
    opts = capi.raster_opts(tile=tile, sh_degree=sh, bg=bg)
    k = oracle.consts(tile=tile, sh_degree=sh)
    rz = Rasterizer("cuda", opts)
    params = G.gpu_params(g)
    gcam = G.gpu_camera(cam)
    fr = rz.forward(params, g.shape[0], gcam, examined=True)
    torch.cuda.synchronize()
    return rz, params, gcam, fr, k, G.oracle_camera(cam), G.f32(g), G.f32(bg)


def _records(rz, P):
    feat = G.np_(rz.feat[:P]).astype(np.float64)
    return dict(feat=feat[:, :9], uv=feat[:, :2], radius=G.np_(rz.radius[:P]),
                key=G.np_(rz.depth[:P]).view(np.uint32), tiles=G.np_(rz.tiles[:P]),
                clamp=G.np_(rz.clamp[:P]))


def _gpu_bins(rz, fr):
    gid = G.np_(rz.gid[: fr.M]).view(np.uint32)
    ranges = G.np_(rz.ranges[: rz.n_tiles]).view(np.uint32)
    return gid, ranges


def _three_sqrt_lambda(feat):
    """3 sqrt(lambda_max) of the 2D covariance whose inverse is the conic."""
    A, B, C = feat[:, 2], feat[:, 3], feat[:, 4]
    det = A * C - B * B
    s00, s01, s11 = C / det, -B / det, A / det
    return 3.0 * np.sqrt(0.5 * (s00 + s11) + np.sqrt(0.25 * (s00 - s11) ** 2 + s01 ** 2))


# ---------------------------------------------------------------- config 0
@pytest.fixture(scope="module")
def cfg0():
    g, cam, target = U.cfg0_scene()
    return g, cam, target


def test_cfg0_projection(cfg0):
    g, cam, _ = cfg0
    rz, params, gcam, fr, k, ocam, g64, _ = _setup(g, cam)
    rec = _records(rz, g.shape[0])
    pr = oracle.project(g64, ocam, k)
    vis = pr["radius"] > 0
    assert vis.sum() > 500
    np.testing.assert_array_equal(rec["radius"] > 0, vis)
    f, fo = rec["feat"][vis], pr["feat"][vis]
    np.testing.assert_allclose(f[:, :2], fo[:, :2], rtol=1e-5, atol=1e-4)
    cn = np.abs(fo[:, 2:5]).max(axis=1, keepdims=True)
    assert np.all(np.abs(f[:, 2:5] - fo[:, 2:5]) <= 1e-4 * cn)
    np.testing.assert_allclose(f[:, 5], fo[:, 5], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(f[:, 6:9], fo[:, 6:9], atol=1e-5)
    np.testing.assert_allclose(G.np_(rz.depth[: g.shape[0]]), pr["depth"], rtol=1e-6)
    # integer outputs: radius = ceil(3 sqrt(lambda)) may differ only where the
    # FP64 value sits at a rounding point (within FP32 error of an integer),
    # and then by one
    diff = np.flatnonzero(rec["radius"][vis] != pr["radius"][vis])
    r3 = _three_sqrt_lambda(fo[diff])
    near = np.abs(r3 - np.round(r3)) <= 1e-4 + 2e-5 * r3
    assert near.all(), (diff[~near], r3[~near])
    assert np.all(np.abs(rec["radius"][vis][diff] - pr["radius"][vis][diff]) == 1)
    obits = pr["clamp"][vis].astype(np.int32) @ np.array([1, 2, 4])
    np.testing.assert_array_equal(rec["clamp"][vis], obits)


def test_cfg0_binning_bit_exact(cfg0):
    g, cam, _ = cfg0
    rz, params, gcam, fr, k, ocam, g64, _ = _setup(g, cam)
    rec = _records(rz, g.shape[0])
    ob = oracle.bin_sort(rec["uv"], rec["radius"], rec["key"], 64, 64, 16)
    gid, ranges = _gpu_bins(rz, fr)
    assert fr.M == ob["M"] and fr.M > 1000
    np.testing.assert_array_equal(gid, ob["gid"])
    np.testing.assert_array_equal(ranges, ob["ranges"])
    assert int(rec["tiles"].sum()) == fr.M


@pytest.mark.parametrize("W,H,B", [(64, 64, 16), (197, 131, 8), (197, 131, 16)])
def test_margin_scene_full_fp64_binning_bit_exact(W, H, B):
    """On a scene kept away from every discrete threshold of the binning (u, v
    and 3 sqrt(lambda_max) not within 1e-4 of an integer, depths apart), the
    FP64 oracle's own projection gives the same radii, rects and pair list as
    the FP32 CUDA path, bit for bit (Eq. 1's per-tile depth order)."""
    cam = synth.camera_cfg0(W, H, 4.0)
    k = oracle.consts(tile=B)
    g, _ = U.margin_scene(oracle, 1000, 7 + W + B, G.oracle_camera(cam), k)
    rz, params, gcam, fr, k, ocam, g64, _ = _setup(g, cam, tile=B)
    rec = _records(rz, g.shape[0])
    pr = oracle.project(g64, ocam, k)
    assert np.all(pr["radius"] > 0)
    np.testing.assert_array_equal(rec["radius"], pr["radius"])
    np.testing.assert_array_equal(rec["tiles"], pr["tiles"])
    ob = oracle.bin_sort(pr["feat"][:, :2], pr["radius"], pr["depth_key"], W, H, B)
    gid, ranges = _gpu_bins(rz, fr)
    assert fr.M == ob["M"] and fr.M > 1000
    np.testing.assert_array_equal(gid, ob["gid"])
    np.testing.assert_array_equal(ranges, ob["ranges"])


def test_cfg0_render_given_records(cfg0):
    g, cam, _ = cfg0
    for bg in ((0.0, 0.0, 0.0), (0.25, 0.5, 1.0)):
        rz, params, gcam, fr, k, ocam, g64, bg64 = _setup(g, cam, bg=bg)
        rec = _records(rz, g.shape[0])
        gid, ranges = _gpu_bins(rz, fr)
        orf = oracle.render_fwd(rec["feat"], 64, 64, 16, gid, ranges, bg64, k)
        assert np.abs(G.np_(fr.img) - orf["img"]).max() <= 1e-5
        assert np.abs(G.np_(fr.T) - orf["T"]).max() <= 1e-5
        np.testing.assert_array_equal(G.np_(fr.last), orf["last"])
        np.testing.assert_array_equal(G.np_(rz.examined), orf["examined"])
        np.testing.assert_array_equal(G.np_(rz.blended), orf["blended"])


def test_cfg0_full_image(cfg0):
    g, cam, _ = cfg0
    rz, params, gcam, fr, k, ocam, g64, bg64 = _setup(g, cam)
    of = oracle.forward(g64, ocam, k, bg=bg64)
    err = np.abs(G.np_(fr.img) - of["img"]).max()
    assert err <= 1e-5, err


def test_cfg0_render_bwd_given_records(cfg0):
    g, cam, target = cfg0
    rz, params, gcam, fr, k, ocam, g64, bg64 = _setup(g, cam)
    rec = _records(rz, g.shape[0])
    gid, ranges = _gpu_bins(rz, fr)
    rng = np.random.default_rng(0)
    dL = rng.normal(size=(3, 64, 64)).astype(np.float32) / (3 * 64 * 64)
    grads = torch.empty_like(params)
    rz.backward(params, fr, torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    g2 = G.np_(rz.grad2d[: g.shape[0]])[:, :9]
    og2 = oracle.render_bwd(rec["feat"], 64, 64, 16, gid, ranges, bg64, k, dL.astype(np.float64))
    ok, worst, nbad = G.grad_close(g2, og2)
    assert ok, (worst, nbad)
    # project adjoint given the same 2D gradients
    og = oracle.project_bwd(g64, ocam, k, g2.astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(grads).T, og)
    assert ok, (worst, nbad)


def test_cfg0_full_gradient_through_autograd(cfg0):
    g, cam, target = cfg0
    opts = capi.raster_opts()
    k = oracle.consts()
    rz = Rasterizer("cuda", opts)
    params = G.gpu_params(g).requires_grad_(True)
    img = rasterize(params, rz, G.gpu_camera(cam))
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    # L1 through the library's loss kernel
    n = img.numel()
    dL = torch.empty_like(img)
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(capi.dg_loss_workspace_size(n), dtype=torch.uint8, device="cuda")
    capi.dg_loss_l1(img.detach(), tgt, n, dL, loss, ws, ws.numel())
    img.backward(dL)
    torch.cuda.synchronize()
    g64 = G.f32(g)
    ocam = G.oracle_camera(cam)
    of = oracle.forward(g64, ocam, k)
    oloss, odL = oracle.loss_l1(of["img"], G.f32(target))
    assert abs(loss.item() - oloss) <= 1e-6
    # the sign pattern of dL/dimg decides the gradient: compare with the oracle's
    # backward fed the GPU's dL (ties |I - target| < 1e-5 may flip)
    flips = np.sign(G.np_(dL)) != np.sign(odL)
    assert flips.mean() < 1e-3
    np.testing.assert_allclose(G.np_(dL)[~flips], odL[~flips], rtol=1e-7)
    ob = oracle.backward(g64, ocam, k, of, G.np_(dL).astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(params.grad).T, ob["grad"])
    assert ok, (worst, nbad)


# ---------------------------------------------------------------- shapes, tiles
@pytest.mark.parametrize("W,H,tile,n", [(72, 40, 16, 3000), (50, 37, 8, 2000), (16, 16, 16, 50),
                                        (200, 130, 16, 20000)])
def test_ragged_sizes_and_tile8(W, H, tile, n):
    g = synth.random_gaussians(n, 77 + n)
    g[:, 3:6] += 0.4
    cam = synth.camera_cfg0(W, H, 4.0)
    bg = (0.1, 0.2, 0.3)
    rz, params, gcam, fr, k, ocam, g64, bg64 = _setup(g, cam, bg=bg, tile=tile)
    rec = _records(rz, n)
    ob = oracle.bin_sort(rec["uv"], rec["radius"], rec["key"], W, H, tile)
    gid, ranges = _gpu_bins(rz, fr)
    np.testing.assert_array_equal(gid, ob["gid"])
    np.testing.assert_array_equal(ranges, ob["ranges"])
    orf = oracle.render_fwd(rec["feat"], W, H, tile, gid, ranges, bg64, k)
    assert np.abs(G.np_(fr.img) - orf["img"]).max() <= 1e-5
    np.testing.assert_array_equal(G.np_(fr.last), orf["last"])
    rng = np.random.default_rng(1)
    dL = (rng.normal(size=(3, H, W)) / (3 * H * W)).astype(np.float32)
    grads = torch.empty_like(params)
    rz.backward(params, fr, torch.from_numpy(dL).cuda(), grads)
    og2 = oracle.render_bwd(rec["feat"], W, H, tile, gid, ranges, bg64, k, dL.astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(rz.grad2d[:n])[:, :9], og2)
    assert ok, (worst, nbad)


@pytest.mark.parametrize("ppt", [1, 2, 4])
@pytest.mark.parametrize("W,H", [(64, 64), (72, 40), (130, 99)])
def test_pixels_per_thread_variants(ppt, W, H):
    g = synth.random_gaussians(4000, 5 + W)
    g[:, 3:6] += 0.3
    cam = synth.camera_cfg0(W, H, 4.0)
    bg = (0.3, 0.1, 0.2)
    opts = capi.raster_opts(bg=bg)
    k = oracle.consts()
    rz = Rasterizer("cuda", opts, ppt_fwd=ppt, ppt_bwd=ppt)
    params = G.gpu_params(g)
    fr = rz.forward(params, g.shape[0], G.gpu_camera(cam), examined=True)
    torch.cuda.synchronize()
    rec = _records(rz, g.shape[0])
    gid, ranges = _gpu_bins(rz, fr)
    orf = oracle.render_fwd(rec["feat"], W, H, 16, gid, ranges, G.f32(bg), k)
    assert np.abs(G.np_(fr.img) - orf["img"]).max() <= 1e-5
    np.testing.assert_array_equal(G.np_(fr.last), orf["last"])
    np.testing.assert_array_equal(G.np_(rz.examined), orf["examined"])
    np.testing.assert_array_equal(G.np_(rz.blended), orf["blended"])
    rng = np.random.default_rng(ppt)
    dL = (rng.normal(size=(3, H, W)) / (3 * H * W)).astype(np.float32)
    grads = torch.empty_like(params)
    rz.backward(params, fr, torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    og2 = oracle.render_bwd(rec["feat"], W, H, 16, gid, ranges, G.f32(bg), k, dL.astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(rz.grad2d[: g.shape[0]])[:, :9], og2)
    assert ok, (worst, nbad)


def test_batched_views_with_many_culled_records():
    """Views that each cull thousands of records: batched binning must equal
    per-view binning (pair lists, ranges) and the oracle's order."""
    g = synth.random_gaussians(20000, 77)
    g[:, 0:3] *= 3.0  # spread beyond every view's frustum
    sizes = [(40, 30), (48, 32), (40, 30), (56, 24), (40, 30), (32, 40)]
    cams = [synth.camera_cfg0(W, H, 3.0 + 0.2 * i) for i, (W, H) in enumerate(sizes)]
    P = g.shape[0]
    params = G.gpu_params(g)
    gcams = [G.gpu_camera(c) for c in cams]
    opts = capi.raster_opts(tile=8)
    rzb = Rasterizer("cuda", opts)
    frb = rzb.forward(params, P, gcams)
    torch.cuda.synchronize()
    assert int(G.np_(rzb.status)[0]) == 0
    radius = G.np_(rzb.radius[: len(sizes) * P]).reshape(len(sizes), P)
    assert ((radius == 0).sum(axis=1) > 4096).all()  # more culled records per view than one emit window
    gid = G.np_(rzb.gid[: frb.M]).view(np.uint32)
    ranges = G.np_(rzb.ranges[: rzb.n_tiles]).view(np.uint32)
    t0 = 0
    for v, (c, (W, H)) in enumerate(zip(gcams, sizes)):
        rz = Rasterizer("cuda", opts)
        fr = rz.forward(params, P, c)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(G.np_(frb.images[v]), G.np_(fr.img))
        nt = ((W + 7) // 8) * ((H + 7) // 8)
        rg = ranges[t0: t0 + nt]
        gid1 = G.np_(rz.gid[: fr.M]).view(np.uint32)
        rg1 = G.np_(rz.ranges[:nt]).view(np.uint32)
        for t in range(nt):
            np.testing.assert_array_equal(gid[rg[t, 0]: rg[t, 1]] - v * P, gid1[rg1[t, 0]: rg1[t, 1]])
        t0 += nt


# ---------------------------------------------------------------- split lists
def _render_split(g, cam, tile, split, bg, ppt=None):
    opts = capi.raster_opts(tile=tile, bg=bg, split_len=split)
    rz = Rasterizer("cuda", opts, ppt_fwd=ppt, ppt_bwd=ppt)
    params = G.gpu_params(g)
    fr = rz.forward(params, g.shape[0], G.gpu_camera(cam), examined=True)
    torch.cuda.synchronize()
    return rz, params, fr


@pytest.mark.parametrize("tile,ppt", [(8, None), (8, 2), (16, 1), (16, 2), (16, 4)])
@pytest.mark.parametrize("split", [-1, 0, 16, 37, 100])
def test_split_lists_match_oracle(tile, ppt, split):
    """Chunked compositing (product pass, exact pass from the prefix product,
    combine) gives the sequential Eq. 1 result: same last/examined/blended,
    images and gradients within tolerance, for chunk lengths that do and do
    not divide the batch size."""
    W, H, n = 130, 99, 6000
    g = synth.random_gaussians(n, 4242)
    g[:, 3:6] += 0.3
    cam = synth.camera_cfg0(W, H, 4.0)
    bg = (0.3, 0.1, 0.2)
    rz, params, fr = _render_split(g, cam, tile, split, bg, ppt)
    k = oracle.consts(tile=tile)
    rec = _records(rz, n)
    gid, ranges = _gpu_bins(rz, fr)
    orf = oracle.render_fwd(rec["feat"], W, H, tile, gid, ranges, G.f32(bg), k)
    assert np.abs(G.np_(fr.img) - orf["img"]).max() <= 1e-5
    assert np.abs(G.np_(fr.T) - orf["T"]).max() <= 1e-5
    np.testing.assert_array_equal(G.np_(fr.last), orf["last"])
    np.testing.assert_array_equal(G.np_(rz.examined), orf["examined"])
    np.testing.assert_array_equal(G.np_(rz.blended), orf["blended"])
    rng = np.random.default_rng(11)
    dL = (rng.normal(size=(3, H, W)) / (3 * H * W)).astype(np.float32)
    grads = torch.empty_like(params)
    rz.backward(params, fr, torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    og2 = oracle.render_bwd(rec["feat"], W, H, tile, gid, ranges, G.f32(bg), k, dL.astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(rz.grad2d[:n])[:, :9], og2)
    assert ok, (worst, nbad)


def test_split_low_resolution_long_lists():
    """A low-resolution view of many Gaussians (thousands of entries per
    tile, many pixels never reaching the stop threshold): automatic
    splitting vs no splitting vs the oracle."""
    W, H, n = 61, 41, 30000
    g = synth.random_gaussians(n, 999)
    g[:, 10] = -1.5  # low opacity: long compositing chains
    cam = synth.camera_cfg0(W, H, 4.0)
    bg = (0.0, 0.0, 0.0)
    out = {}
    for split in (-1, 0):
        rz, params, fr = _render_split(g, cam, 8, split, bg)
        rng = np.random.default_rng(5)
        dL = (rng.normal(size=(3, H, W)) / (3 * H * W)).astype(np.float32)
        grads = torch.empty_like(params)
        rz.backward(params, fr, torch.from_numpy(dL).cuda(), grads)
        torch.cuda.synchronize()
        out[split] = (rz, fr, dL, G.np_(rz.grad2d[:n])[:, :9].copy(), G.np_(grads))
    rz, fr, dL, g2, _ = out[0]
    rz1, fr1, _, g21, _ = out[-1]
    assert int(G.np_(rz.examined).max()) > 1000  # long chains are exercised
    np.testing.assert_array_equal(G.np_(fr.last), G.np_(fr1.last))
    np.testing.assert_array_equal(G.np_(rz.examined), G.np_(rz1.examined))
    np.testing.assert_array_equal(G.np_(rz.blended), G.np_(rz1.blended))
    assert np.abs(G.np_(fr.img) - G.np_(fr1.img)).max() <= 1e-5
    k = oracle.consts(tile=8)
    rec = _records(rz, n)
    gid, ranges = _gpu_bins(rz, fr)
    orf = oracle.render_fwd(rec["feat"], W, H, 8, gid, ranges, np.zeros(3), k)
    assert np.abs(G.np_(fr.img) - orf["img"]).max() <= 1e-5
    np.testing.assert_array_equal(G.np_(fr.last), orf["last"])
    og2 = oracle.render_bwd(rec["feat"], W, H, 8, gid, ranges, np.zeros(3), k, dL.astype(np.float64))
    for got in (g2, g21):
        ok, worst, nbad = G.grad_close(got, og2)
        assert ok, (worst, nbad)


@pytest.mark.parametrize("tile", [8, 16])
def test_binning_many_tiles_with_depth_ties(tile):
    """Depth order over 30 radix tiles plus a ragged tail, with most keys tied:
    two exact planes (every Gaussian of a plane has the same depth bits, so
    only stability across tiles puts them in index order), a few scattered
    depths, some Gaussians behind the camera and some off-screen.  The lists
    must equal the oracle's (tile, depth bits, index) order bit for bit."""
    rng = np.random.default_rng(77)
    W, H, f = 320, 200, 200.0
    P = 30 * 2048 + 1001
    z = np.where(rng.random(P) < 0.45, 3.0, 5.0)
    scatter = rng.random(P) < 0.1
    z[scatter] = rng.uniform(2.0, 8.0, size=int(scatter.sum()))
    behind = rng.random(P) < 0.05
    z[behind] = -1.0
    u = rng.uniform(-10.0, W + 10.0, size=P)
    v = rng.uniform(-10.0, H + 10.0, size=P)
    off = rng.random(P) < 0.05
    u[off] += 5000.0
    g = np.zeros((P, synth.NPARAM))
    g[:, 0] = (u - W / 2) * z / f
    g[:, 1] = (v - H / 2) * z / f
    g[:, 2] = z
    g[:, 3:6] = rng.normal(-4.0, 0.3, size=(P, 3))
    g[:, 6] = 1.0
    g[:, 10] = 0.5
    cam = U.identity_cam(W, H, f)
    rz, params, gcam, fr, k, ocam, g64, _ = _setup(g, cam, tile=tile)
    rec = _records(rz, P)
    vis = rec["radius"] > 0
    keys = rec["key"][vis]
    assert vis.sum() > 40000 and (~vis).sum() > 1000
    assert len(keys) - len(np.unique(keys)) > 30000  # most keys are ties
    ob = oracle.bin_sort(rec["uv"], rec["radius"], rec["key"], W, H, tile)
    gid, ranges = _gpu_bins(rz, fr)
    assert fr.M == ob["M"] == int(rec["tiles"].sum())
    np.testing.assert_array_equal(gid, ob["gid"])
    np.testing.assert_array_equal(ranges, ob["ranges"])


def test_empty_and_all_culled():
    cam = U.identity_cam(40, 24, 50.0)
    bg = (0.2, 0.5, 0.9)
    for g in (np.zeros((0, 59)),
              np.concatenate([U.single_gaussian((0, 0, 0.1), [-2] * 3), U.single_gaussian((0, 0, -3.0), [-2] * 3)])):
        opts = capi.raster_opts(bg=bg)
        rz = Rasterizer("cuda", opts)
        params = G.gpu_params(g) if g.shape[0] else torch.zeros((59, 0), device="cuda")
        fr = rz.forward(params, g.shape[0], G.gpu_camera(cam))
        torch.cuda.synchronize()
        assert fr.M == 0
        img = G.np_(fr.img)
        for c in range(3):
            assert np.all(img[c] == np.float32(bg[c]))
        assert np.all(G.np_(fr.T) == 1.0) and np.all(G.np_(fr.last) == 0)


def test_pair_capacity_overflow_reports_status():
    g, cam, _ = U.cfg0_scene()
    opts = capi.raster_opts()
    rz = Rasterizer("cuda", opts)
    params = G.gpu_params(g)
    gcam = G.gpu_camera(cam)
    fr = rz.forward(params, g.shape[0], gcam)
    P = g.shape[0]
    M = fr.M
    small = M // 2
    ws = torch.empty(capi.dg_bin_workspace_size(P, 1, small), dtype=torch.uint8, device="cuda")
    gid = torch.full((small,), -7, dtype=torch.int32, device="cuda")
    ranges = torch.full((rz.n_tiles, 2), 5, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    Mdev = torch.zeros(1, dtype=torch.int64, device="cuda")
    capi.dg_bin_count(rz.depth, rz.tiles, P, 1, ws, ws.numel(), small, Mdev)
    capi.dg_bin_sort(rz.feat, rz.radius, P, gcam, 1, 16, ws, ws.numel(), small, gid, ranges, status)
    torch.cuda.synchronize()
    assert int(Mdev.item()) == M
    assert int(status.item()) == capi.DG_ERR_CAPACITY
    assert bool((gid == -7).all()) and bool((ranges == 0).all())


def test_host_side_argument_errors():
    opts = capi.raster_opts(sh_degree=5)
    cam = G.gpu_camera(synth.camera_cfg0(64, 64, 4.0))
    t = torch.zeros((59, 4), device="cuda")
    with pytest.raises(capi.DashGSError) as e:
        capi.dg_project(t, 4, 4, cam, 1, opts, t, t, t, t, t)
    assert e.value.status == capi.DG_ERR_ARG and "sh_degree" in str(e.value)
    with pytest.raises(capi.DashGSError):
        capi.dg_project(t, 2, 4, cam, 1, capi.raster_opts(), t, t, t, t, t)  # stride < P


# ---------------------------------------------------------------- loss, Adam
def test_loss_l1_parity():
    rng = np.random.default_rng(5)
    a = rng.uniform(size=(3, 41, 57)).astype(np.float32)
    b = rng.uniform(size=(3, 41, 57)).astype(np.float32)
    b[0, :3, :3] = a[0, :3, :3]
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    n = a.size
    d = torch.empty_like(ta)
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(capi.dg_loss_workspace_size(n), dtype=torch.uint8, device="cuda")
    capi.dg_loss_l1(ta, tb, n, d, loss, ws, ws.numel())
    torch.cuda.synchronize()
    ol, og = oracle.loss_l1(a.astype(np.float64), b.astype(np.float64))
    assert abs(loss.item() - ol) <= 1e-6 * ol
    np.testing.assert_array_equal(G.np_(d), og.astype(np.float32))


def test_adam_parity():
    rng = np.random.default_rng(6)
    P = 1000 + 3  # ragged tail beyond the 4-wide vector path
    stride = 1010
    p = rng.normal(size=(59, stride)).astype(np.float32)
    lr = np.linspace(1e-4, 1e-2, 59).astype(np.float32)
    tp = torch.from_numpy(p.copy()).cuda()
    m = torch.zeros_like(tp); v = torch.zeros_like(tp)
    op = p[:, :P].astype(np.float64).copy(); om = np.zeros_like(op); ov = np.zeros_like(op)
    for step in range(1, 6):
        gr = rng.normal(size=(59, stride)).astype(np.float32)
        capi.dg_adam_step(tp, torch.from_numpy(gr).cuda(), m, v, stride, P, lr, 0.9, 0.999, 1e-15, step)
        oracle.adam(op, gr[:, :P].astype(np.float64), om, ov, np.broadcast_to(lr[:, None].astype(np.float64), op.shape).copy(),
                    0.9, 0.999, 1e-15, step)
    torch.cuda.synchronize()
    got = G.np_(tp)
    np.testing.assert_allclose(got[:, :P], op, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(got[:, P:], p[:, P:])  # padding untouched


@pytest.mark.parametrize("sh,V,trim,pad", [(3, 1, 0, 13), (2, 1, 0, 13), (0, 1, 0, 13), (3, 3, 0, 13), (1, 2, 0, 13),
                                          (3, 1, 0, 0), (3, 1, 2, 2), (1, 2, 3, 7)])
def test_fused_project_bwd_adam_matches_two_calls(sh, V, trim, pad):
    """dg_project_bwd_adam = dg_project_bwd followed by dg_adam_step
    (including Gaussians culled in every view, whose moments still decay).
    The adjoint's two instantiations may contract multiply-adds differently,
    so their gradients agree within the gradient tolerance; the Adam update is
    one contraction-free function, so given the same gradient the state is
    bit-identical.  Row strides P + pad: a multiple of 4 (16-byte row accesses
    in the fused sweep, with P - trim leaving lanes at the end of P) or not
    (4-byte accesses); columns from P on stay untouched."""
    g = synth.random_gaussians(3000, 21 + V)[: 3000 - trim]
    g[:, 3:6] += 0.3
    g[-50:, 0] = 100.0  # off-screen in every view: culled, zero gradient, moments still decay
    sizes = [(64, 64), (90, 50), (40, 70)][:V]
    cams = [G.gpu_camera(synth.camera_cfg0(W, H, 4.0 + 0.7 * i)) for i, (W, H) in enumerate(sizes)]
    opts = capi.raster_opts(sh_degree=sh)
    rz = Rasterizer("cuda", opts)
    P = g.shape[0]
    stride = P + pad
    base = np.zeros((59, stride), np.float32)
    base[:, :P] = g.T
    params = torch.from_numpy(base).cuda()
    fr = rz.forward(params[:, :P], P, cams)
    rng = np.random.default_rng(V)
    dL = torch.from_numpy((rng.normal(size=fr.flat_img.numel()) / 1e4).astype(np.float32)).cuda()
    rz.backward(params[:, :P], fr, dL, torch.empty_like(params[:, :P]))
    lr = np.linspace(1e-4, 1e-2, 59).astype(np.float32)
    m0 = torch.from_numpy(rng.normal(size=(59, stride)).astype(np.float32) * 1e-3).cuda()
    v0 = torch.from_numpy(np.abs(rng.normal(size=(59, stride))).astype(np.float32) * 1e-6).cuda()
    # two calls
    p1, m1, v1 = params.clone(), m0.clone(), v0.clone()
    grads = torch.zeros_like(params)
    capi.dg_project_bwd(p1, stride, P, cams, V, opts, rz.radius, rz.clamp, rz.grad2d, grads)
    capi.dg_adam_step(p1, grads, m1, v1, stride, P, lr, 0.9, 0.999, 1e-15, 7)
    # fused, also writing the gradient
    p2, m2, v2 = params.clone(), m0.clone(), v0.clone()
    grads2 = torch.zeros_like(params)
    capi.dg_project_bwd_adam(p2, stride, P, cams, V, opts, rz.radius, rz.clamp, rz.grad2d, grads2, m2, v2, lr, 0.9,
                             0.999, 1e-15, 7)
    torch.cuda.synchronize()
    ok, worst, nbad = G.grad_close(G.np_(grads2), G.np_(grads))
    assert ok, (worst, nbad)
    p4, m4, v4 = params.clone(), m0.clone(), v0.clone()
    capi.dg_adam_step(p4, grads2, m4, v4, stride, P, lr, 0.9, 0.999, 1e-15, 7)
    torch.cuda.synchronize()
    for a, b in ((p2, p4), (m2, m4), (v2, v4)):
        np.testing.assert_array_equal(G.np_(a), G.np_(b))
    assert (G.np_(rz.radius[: V * P]).reshape(V, P) == 0).all(axis=0).any()  # some Gaussians culled everywhere
    # without the gradient output
    p3, m3, v3 = params.clone(), m0.clone(), v0.clone()
    capi.dg_project_bwd_adam(p3, stride, P, cams, V, opts, rz.radius, rz.clamp, rz.grad2d, None, m3, v3, lr, 0.9,
                             0.999, 1e-15, 7)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(G.np_(p3), G.np_(p2))


def test_fused_project_bwd_adam_device_hparams_and_skip():
    """dg_project_bwd_adam_dev (hyper-parameters read from device memory, as a
    replayed CUDA graph does) gives the bits of dg_project_bwd_adam with the
    same values; with the skip word set it leaves params, m and v untouched
    and still writes the gradient."""
    import ctypes
    g = synth.random_gaussians(2000, 77)
    g[:, 3:6] += 0.3
    cams = [G.gpu_camera(synth.camera_cfg0(64, 64, 4.0))]
    opts = capi.raster_opts(sh_degree=3)
    rz = Rasterizer("cuda", opts)
    P = g.shape[0]
    stride = P + 5
    base = np.zeros((59, stride), np.float32)
    base[:, :P] = g.T
    params = torch.from_numpy(base).cuda()
    fr = rz.forward(params[:, :P], P, cams)
    rng = np.random.default_rng(3)
    dL = torch.from_numpy((rng.normal(size=fr.flat_img.numel()) / 1e4).astype(np.float32)).cuda()
    rz.backward(params[:, :P], fr, dL, torch.empty_like(params[:, :P]))
    lr = np.linspace(1e-4, 1e-2, 59).astype(np.float32)
    m0 = torch.from_numpy(rng.normal(size=(59, stride)).astype(np.float32) * 1e-3).cuda()
    v0 = torch.from_numpy(np.abs(rng.normal(size=(59, stride))).astype(np.float32) * 1e-6).cuda()
    p1, m1, v1 = params.clone(), m0.clone(), v0.clone()
    capi.dg_project_bwd_adam(p1, stride, P, cams, 1, opts, rz.radius, rz.clamp, rz.grad2d, None, m1, v1, lr, 0.9,
                             0.999, 1e-15, 9)
    hp = capi.dg_adam_hparams_fill(lr, 0.9, 0.999, 1e-15, 9)
    raw = np.frombuffer(ctypes.string_at(ctypes.addressof(hp), ctypes.sizeof(hp)), dtype=np.uint8).copy()
    hp_dev = torch.from_numpy(raw).cuda()
    p2, m2, v2 = params.clone(), m0.clone(), v0.clone()
    capi.dg_project_bwd_adam_dev(p2, stride, P, cams, 1, opts, rz.radius, rz.clamp, rz.grad2d, None, m2, v2, hp_dev,
                                 skip_if=torch.zeros(1, dtype=torch.int32, device="cuda"))
    p3, m3, v3 = params.clone(), m0.clone(), v0.clone()
    grads3 = torch.zeros_like(params)
    capi.dg_project_bwd_adam_dev(p3, stride, P, cams, 1, opts, rz.radius, rz.clamp, rz.grad2d, grads3, m3, v3, hp_dev,
                                 skip_if=torch.full((1,), -2, dtype=torch.int32, device="cuda"))
    grads4 = torch.zeros_like(params)
    capi.dg_project_bwd(params, stride, P, cams, 1, opts, rz.radius, rz.clamp, rz.grad2d, grads4)
    torch.cuda.synchronize()
    for a, b in ((p1, p2), (m1, m2), (v1, v2)):
        np.testing.assert_array_equal(G.np_(a), G.np_(b))
    for a, b in ((p3, params), (m3, m0), (v3, v0)):
        np.testing.assert_array_equal(G.np_(a), G.np_(b))
    assert float(grads3.abs().max()) > 0.0
    ok, worst, nbad = G.grad_close(G.np_(grads3), G.np_(grads4))
    assert ok, (worst, nbad)


# ---------------------------------------------------------------- full size, sampled
@pytest.fixture(scope="module")
def fullsize():
    """The bench's workload: 2M-Gaussian textured scene, one 1237x822 view."""
    gt = synth.textured_scene(2_000_000, 1001)
    model = synth.jitter(gt, 3001)
    view = synth.ring_cameras(160, 1237, 822, 5.0, 2001)[0]
    rz = Rasterizer("cuda", capi.raster_opts())
    params = G.gpu_params(model)
    gcam = G.gpu_camera(view)
    fr = rz.forward(params, model.shape[0], gcam, examined=True)
    torch.cuda.synchronize()
    return model, view, rz, params, gcam, fr


def test_fullsize_sampled_tiles_and_pixels(fullsize):
    model, view, rz, params, gcam, fr = fullsize
    P, W, H = model.shape[0], 1237, 822
    rec = _records(rz, P)
    gid, ranges = _gpu_bins(rz, fr)
    assert fr.M > 2_000_000 and int(rec["tiles"].sum()) == fr.M
    # ranges partition [0, M) in tile order
    nz = ranges[:, 1] > ranges[:, 0]
    assert ranges[nz, 0].min() == 0 and ranges[nz, 1].max() == fr.M
    assert int((ranges[:, 1] - ranges[:, 0]).sum()) == fr.M
    rng = np.random.default_rng(7)
    n_tiles = ranges.shape[0]
    tiles = np.concatenate([[0, n_tiles - 1, 77], rng.choice(n_tiles, 21, replace=False)])
    k = oracle.consts()
    for t in tiles:
        ref = oracle.tile_list(rec["uv"], rec["radius"], rec["key"], W, H, 16, int(t))
        s, e = ranges[t]
        np.testing.assert_array_equal(gid[s:e], ref)
    # sampled pixels (including the ragged last row/column) against Eq. 1
    px = np.concatenate([[0, W - 1, W - 1, 0], rng.integers(0, W, 300)])
    py = np.concatenate([[0, 0, H - 1, H - 1], rng.integers(0, H, 300)])
    o = oracle.render_pixels(rec["feat"], W, 16, gid, ranges, np.zeros(3), k, px, py)
    img = G.np_(fr.img)
    assert np.abs(img[:, py, px].T - o["rgb"]).max() <= 1e-5
    assert np.abs(G.np_(fr.T)[py, px] - o["T"]).max() <= 1e-5
    np.testing.assert_array_equal(G.np_(fr.last)[py, px], o["last"])
    np.testing.assert_array_equal(G.np_(rz.examined)[py, px], o["examined"])


@pytest.mark.parametrize("tile", [16, 8])
def test_fullsize_backward_on_sampled_tiles(fullsize, tile):
    """The bench's view (tile 16, and tile 8, the bench's launch shape with the
    entry-parallel backward) on tiles of 16x16 pixels with dL/dimg set."""
    model, view, rz, params, gcam, fr = fullsize
    P, W, H = model.shape[0], 1237, 822
    if tile != 16:
        rz = Rasterizer("cuda", capi.raster_opts(tile=tile))
        fr = rz.forward(params, P, gcam)
        torch.cuda.synchronize()
    rec = _records(rz, P)
    gid, ranges = _gpu_bins(rz, fr)
    # dL/dimg non-zero only on a few 16x16 blocks: the oracle's adjoint then touches only them
    rng = np.random.default_rng(8)
    dL = np.zeros((3, H, W), np.float32)
    TX, TY = (W + 15) // 16, (H + 15) // 16
    for t in rng.choice(TX * TY, 6, replace=False):
        ty, tx = divmod(int(t), TX)
        ys, xs = slice(ty * 16, min(H, ty * 16 + 16)), slice(tx * 16, min(W, tx * 16 + 16))
        hh, ww = ys.stop - ys.start, xs.stop - xs.start
        dL[:, ys, xs] = rng.normal(size=(3, hh, ww)).astype(np.float32) / (3 * 64 * 64)
    grads = torch.empty_like(params)
    rz.backward(params, fr, torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    g2 = G.np_(rz.grad2d[:P])[:, :9]
    og2 = oracle.render_bwd(rec["feat"], W, H, tile, gid, ranges, np.zeros(3), oracle.consts(tile=tile),
                            dL.astype(np.float64))
    # same dL normalisation and tolerance as the 64x64 cases (1e-4 relative, 1e-6 absolute)
    ok, worst, nbad = G.grad_close(g2, og2)
    assert ok, (worst, nbad)
    touched = np.abs(og2).sum(1) > 0
    assert touched.sum() > 1000


# ---------------------------------------------------------------- several views per call
def test_batched_views_match_single_view_renders():
    g = synth.random_gaussians(3000, 31)
    g[:, 3:6] += 0.3
    sizes = [(64, 64), (72, 40), (130, 99)]
    cams = []
    for i, (W, H) in enumerate(sizes):
        c = synth.camera_cfg0(W, H, 4.0 + 0.5 * i)
        cams.append(c)
    opts = capi.raster_opts(bg=(0.1, 0.3, 0.2))
    params = G.gpu_params(g)
    P = g.shape[0]
    gcams = [G.gpu_camera(c) for c in cams]
    rzb = Rasterizer("cuda", opts)
    frb = rzb.forward(params, P, gcams, examined=True)
    rng = np.random.default_rng(3)
    dLs = [(rng.normal(size=(3, H, W)) / (3 * 64 * 64)).astype(np.float32) for W, H in sizes]
    dL = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dLs])).cuda()
    gb = torch.empty_like(params)
    rzb.backward(params, frb, dL, gb)
    torch.cuda.synchronize()
    gsum = np.zeros((59, P))
    for v, (c, (W, H)) in enumerate(zip(gcams, sizes)):
        rz = Rasterizer("cuda", opts)
        fr = rz.forward(params, P, c, examined=True)
        gv = torch.empty_like(params)
        rz.backward(params, fr, torch.from_numpy(dLs[v]).cuda(), gv)
        torch.cuda.synchronize()
        # the batched render of a view is the single-view render, bit for bit
        np.testing.assert_array_equal(G.np_(frb.images[v]), G.np_(fr.img))
        np.testing.assert_array_equal(G.np_(frb.Ts[v]), G.np_(fr.T))
        np.testing.assert_array_equal(G.np_(frb.lasts[v]), G.np_(fr.last))
        np.testing.assert_array_equal(G.np_(rzb.blended[v]), G.np_(rz.blended))
        gsum += G.np_(gv)
    ok, worst, nbad = G.grad_close(G.np_(gb).T, gsum.T)
    assert ok, (worst, nbad)
    # and each batched view against the oracle, fed the batch's own FP32
    # records (payload v*P + i) and its pair list; tile ranges of view v
    # start after the tiles of views 0..v-1
    k = oracle.consts()
    feat = G.np_(rzb.feat[: len(sizes) * P]).astype(np.float64)[:, :9]
    gid = G.np_(rzb.gid[: frb.M]).view(np.uint32)
    ranges = G.np_(rzb.ranges[: rzb.n_tiles]).view(np.uint32)
    t0 = 0
    for v, (W, H) in enumerate(sizes):
        nt = ((W + 15) // 16) * ((H + 15) // 16)
        orf = oracle.render_fwd(feat, W, H, 16, gid, ranges[t0: t0 + nt], G.f32((0.1, 0.3, 0.2)), k)
        t0 += nt
        assert np.abs(G.np_(frb.images[v]) - orf["img"]).max() <= 1e-5
        assert np.abs(G.np_(frb.Ts[v]) - orf["T"]).max() <= 1e-5
        np.testing.assert_array_equal(G.np_(frb.lasts[v]), orf["last"])
        np.testing.assert_array_equal(G.np_(rzb.blended[v]), orf["blended"])


def test_max_views_per_call():
    """DG_MAX_VIEWS (16) views in one call, the largest batch: each view's
    render equals its single-view render bit for bit, the summed parameter
    gradient equals the sum of the single-view gradients, the fused adjoint +
    Adam equals the two calls; a 17th view is rejected before any launch."""
    V = 16
    g = synth.random_gaussians(4000, 41)
    g[:, 3:6] += 0.3
    g[-40:, 0] = 100.0  # culled in every view
    sizes = [(40 + 8 * (i % 4), 30 + 5 * (i % 3)) for i in range(V)]
    cams = [G.gpu_camera(synth.camera_cfg0(W, H, 3.5 + 0.15 * i)) for i, (W, H) in enumerate(sizes)]
    # (lists never split: the automatic rule splits the small single-view
    # batches and not the 16-view one, which changes the rounding order)
    opts = capi.raster_opts(tile=8, bg=(0.1, 0.2, 0.3), split_len=-1)
    P = g.shape[0]
    params = G.gpu_params(g)
    rzb = Rasterizer("cuda", opts)
    frb = rzb.forward(params, P, cams)
    rng = np.random.default_rng(16)
    dLs = [(rng.normal(size=(3, H, W)) / (3 * 40 * 30)).astype(np.float32) for W, H in sizes]
    dL = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dLs])).cuda()
    gb = torch.empty_like(params)
    rzb.backward(params, frb, dL, gb)
    torch.cuda.synchronize()
    assert int(G.np_(rzb.status)[0]) == 0
    gsum = np.zeros((59, P))
    for v in range(V):
        rz = Rasterizer("cuda", opts)
        fr = rz.forward(params, P, cams[v])
        gv = torch.empty_like(params)
        rz.backward(params, fr, torch.from_numpy(dLs[v]).cuda(), gv)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(G.np_(frb.images[v]), G.np_(fr.img))
        np.testing.assert_array_equal(G.np_(frb.Ts[v]), G.np_(fr.T))
        np.testing.assert_array_equal(G.np_(frb.lasts[v]), G.np_(fr.last))
        gsum += G.np_(gv)
    ok, worst, nbad = G.grad_close(G.np_(gb).T, gsum.T)
    assert ok, (worst, nbad)
    # the fused multi-view adjoint + Adam against the two calls
    lr = np.linspace(1e-4, 1e-2, 59).astype(np.float32)
    m0 = torch.from_numpy(rng.normal(size=(59, P)).astype(np.float32) * 1e-3).cuda()
    v0 = torch.from_numpy(np.abs(rng.normal(size=(59, P))).astype(np.float32) * 1e-6).cuda()
    p2, m2, v2 = params.clone(), m0.clone(), v0.clone()
    grads2 = torch.zeros_like(params)
    capi.dg_project_bwd_adam(p2, P, P, cams, V, opts, rzb.radius, rzb.clamp, rzb.grad2d, grads2, m2, v2, lr, 0.9,
                             0.999, 1e-15, 3)
    p4, m4, v4 = params.clone(), m0.clone(), v0.clone()
    capi.dg_adam_step(p4, grads2, m4, v4, P, P, lr, 0.9, 0.999, 1e-15, 3)
    torch.cuda.synchronize()
    ok, worst, nbad = G.grad_close(G.np_(grads2).T, G.np_(gb).T)
    assert ok, (worst, nbad)
    for a, b in ((p2, p4), (m2, m4), (v2, v4)):
        np.testing.assert_array_equal(G.np_(a), G.np_(b))
    # one view more than the limit
    cams17 = cams + [cams[0]]
    grads = torch.zeros_like(params)
    with pytest.raises(capi.DashGSError) as e:
        capi.dg_project_bwd(params, P, P, cams17, V + 1, opts, rzb.radius, rzb.clamp, rzb.grad2d, grads)
    assert e.value.status == capi.DG_ERR_ARG
    assert capi.dg_bin_workspace_size(P, V + 1, 1000) == 0


def test_sparse_adam_parity():
    rng = np.random.default_rng(9)
    P, stride = 1003, 1010
    p = rng.normal(size=(59, stride)).astype(np.float32)
    lr = np.linspace(1e-4, 1e-2, 59).astype(np.float32)
    radius = np.where(rng.random((2, P)) < 0.4, rng.integers(1, 9, size=(2, P)), 0).astype(np.int32)
    vis_ref = (radius > 0).any(axis=0)
    vis = torch.zeros(P, dtype=torch.uint8, device="cuda")
    capi.dg_visibility(torch.from_numpy(radius.reshape(-1)).cuda(), P, 2, vis)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(G.np_(vis).astype(bool), vis_ref)
    tp = torch.from_numpy(p.copy()).cuda()
    m = torch.zeros_like(tp); v = torch.zeros_like(tp)
    op = p[:, :P].astype(np.float64).copy(); om = np.zeros_like(op); ov = np.zeros_like(op)
    for step in range(1, 5):
        gr = rng.normal(size=(59, stride)).astype(np.float32)
        capi.dg_sparse_adam_step(tp, torch.from_numpy(gr).cuda(), m, v, stride, P, lr, 0.9, 0.999, 1e-15, step, vis)
        oracle.sparse_adam(op, gr[:, :P].astype(np.float64), om, ov, lr[:, None].astype(np.float64), 0.9, 0.999,
                           1e-15, step, vis_ref)
    torch.cuda.synchronize()
    got = G.np_(tp)
    np.testing.assert_allclose(got[:, :P], op, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(got[:, :P][:, ~vis_ref], p[:, :P][:, ~vis_ref])
    assert float(G.np_(m)[:, :P][:, ~vis_ref].__abs__().max()) == 0.0


def test_mip_2d_filter_matches_oracle():
    """Mip-Splatting's 2D filter (opts.mip2d): records (conic, compensated
    opacity), image and full parameter gradient against the FP64 oracle with
    the same filter."""
    g = synth.random_gaussians(2000, 88)
    g[:, 3:6] -= 1.0  # small footprints: compensation factors well below 1
    cam = synth.camera_cfg0(64, 64, 4.0)
    bg = (0.1, 0.2, 0.3)
    opts = capi.raster_opts(mip2d=0.1, bg=bg)
    k = oracle.consts(mip2d=0.1)
    rz = Rasterizer("cuda", opts)
    params = G.gpu_params(g)
    gcam = G.gpu_camera(cam)
    fr = rz.forward(params, g.shape[0], gcam, examined=True)
    torch.cuda.synchronize()
    rec = _records(rz, g.shape[0])
    g64, ocam = G.f32(g), G.oracle_camera(cam)
    pr = oracle.project(g64, ocam, k)
    vis = pr["radius"] > 0
    assert vis.sum() > 500
    np.testing.assert_array_equal(rec["radius"] > 0, vis)
    f, fo = rec["feat"][vis], pr["feat"][vis]
    assert fo[:, 5].min() < 0.5 * G.np_(torch.sigmoid(params[10]))[vis].max()  # compensation active
    cn = np.abs(fo[:, 2:5]).max(axis=1, keepdims=True)
    assert np.all(np.abs(f[:, 2:5] - fo[:, 2:5]) <= 1e-4 * cn)
    np.testing.assert_allclose(f[:, 5], fo[:, 5], rtol=1e-5, atol=1e-7)
    gid, ranges = _gpu_bins(rz, fr)
    orf = oracle.render_fwd(rec["feat"], 64, 64, 16, gid, ranges, G.f32(bg), k)
    assert np.abs(G.np_(fr.img) - orf["img"]).max() <= 1e-5
    np.testing.assert_array_equal(G.np_(fr.last), orf["last"])
    rng = np.random.default_rng(4)
    dL = (rng.normal(size=(3, 64, 64)) / (3 * 64 * 64)).astype(np.float32)
    grads = torch.empty_like(params)
    rz.backward(params, fr, torch.from_numpy(dL).cuda(), grads)
    torch.cuda.synchronize()
    g2 = G.np_(rz.grad2d[: g.shape[0]])[:, :9]
    og2 = oracle.render_bwd(rec["feat"], 64, 64, 16, gid, ranges, G.f32(bg), k, dL.astype(np.float64))
    ok, worst, nbad = G.grad_close(g2, og2)
    assert ok, (worst, nbad)
    og = oracle.project_bwd(g64, ocam, k, g2.astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(grads).T, og)
    assert ok, (worst, nbad)


def test_backward_with_and_without_blend_flags():
    """The backward stages only entries the forward flagged as blended by some
    pixel of their tile; without room for the flags it falls back to the tile
    test.  Both give the same gradients (only float addition order differs)."""
    g = synth.random_gaussians(5000, 123)
    g[:, 3:6] += 0.2
    cam = G.gpu_camera(synth.camera_cfg0(130, 99, 4.0))
    P = g.shape[0]
    params = G.gpu_params(g)
    out = []
    for with_flags in (True, False):
        rz = Rasterizer("cuda", capi.raster_opts(tile=8))
        fr = rz.forward(params, P, cam)
        if not with_flags:  # re-render into a workspace without the flag bytes
            carr = capi.cameras([cam])
            rz.rws = torch.empty(capi.dg_render_workspace_size(carr, 1, rz.opts_fwd, 0), dtype=torch.uint8,
                                 device="cuda")
            capi.dg_render_fwd(rz.rfeat, rz.gid, rz.ranges, carr, 1, rz.opts_fwd, fr.flat_img, fr.flat_T,
                               fr.flat_last, None, None, rz.rws, rz.rws.numel())
        rng = np.random.default_rng(8)
        dL = torch.from_numpy((rng.normal(size=(3, 99, 130)) / 1e4).astype(np.float32)).cuda()
        rz.backward_render(fr, dL)
        torch.cuda.synchronize()
        out.append(G.np_(rz.grad2d[:P]).copy())
    ok, worst, nbad = G.grad_close(out[0], out[1])
    assert ok, (worst, nbad)
    assert np.abs(out[0]).max() > 0


@pytest.mark.parametrize("ppt_fwd", [1, 2])
def test_tile8_backward_with_per_warp_flags_and_fallback(ppt_fwd):
    """At 8x8 tiles with one pixel per thread the forward writes, per pair,
    which 8x4 block blended the entry, and the backward's warps walk only
    their own block's entries; after a forward at another launch shape (two
    pixels per thread) the flags carry no block bits and every warp walks
    every flagged entry.  Both match the oracle's adjoint (bg != 0, ragged)."""
    g = synth.random_gaussians(6000, 321)
    g[:, 3:6] += 0.25
    W, H = 117, 83
    cam = synth.camera_cfg0(W, H, 4.0)
    bg = (0.2, 0.4, 0.1)
    opts = capi.raster_opts(tile=8, bg=bg)
    rz = Rasterizer("cuda", opts, ppt_fwd=ppt_fwd, ppt_bwd=1)
    P = g.shape[0]
    params = G.gpu_params(g)
    fr = rz.forward(params, P, G.gpu_camera(cam))
    torch.cuda.synchronize()
    rec = _records(rz, P)
    gid, ranges = _gpu_bins(rz, fr)
    k = oracle.consts(tile=8)
    rng = np.random.default_rng(ppt_fwd)
    dL = (rng.normal(size=(3, H, W)) / (3 * H * W)).astype(np.float32)
    rz.backward_render(fr, torch.from_numpy(dL).cuda())
    torch.cuda.synchronize()
    og2 = oracle.render_bwd(rec["feat"], W, H, 8, gid, ranges, G.f32(bg), k, dL.astype(np.float64))
    ok, worst, nbad = G.grad_close(G.np_(rz.grad2d[:P])[:, :9], og2)
    assert ok, (worst, nbad)
    assert np.abs(og2).max() > 0
