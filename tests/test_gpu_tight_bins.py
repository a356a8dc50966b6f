"""Tight pair lists (dg_raster_opts.tight_bins) against the rect lists of the
tile binning (Sec. 2's rasterizer: every tile of a Gaussian's 3-sigma rect).

Checked on the GPU path:
* projection outputs other than the tile mask and count are unchanged;
* every tile's tight list is its rect list with entries left out, in the same
  (depth, index) order;
* every left-out entry fails the alpha >= 1/255 test at every pixel centre of
  its tile inside the image, evaluated in FP64 on the oracle's own records
  (so the paper's compositing never blends it there);
* the compositing passes give the same images and transmittances (bit for
  bit, list splitting off), the same last blended Gaussian per pixel, and the
  same gradients up to the order of float atomics.
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
from tests import _util as U  # noqa: E402

pytestmark = pytest.mark.gpu

ALPHA_MIN = 1.0 / 255.0


def _run(g, cams, tile, tight, record=0, seed=0, mip2d=0.0, bg=(0.0, 0.0, 0.0)):
    """Forward (with per-pixel counts) and full backward of one configuration."""
    opts = capi.raster_opts(tile=tile, sh_degree=3, split_len=-1, record=record, tight_bins=tight, mip2d=mip2d,
                            bg=bg)
    rz = Rasterizer("cuda", opts)
    params = G.gpu_params(g)
    P = g.shape[0]
    gc = [G.gpu_camera(c) for c in cams]
    fr = rz.forward(params, P, gc if len(gc) > 1 else gc[0], examined=True)
    rng = np.random.default_rng(seed)
    dL = torch.from_numpy(rng.normal(size=fr.flat_img.numel()).astype(np.float32)).cuda()
    grads = torch.zeros_like(params)
    rz.backward(params, fr, dL, grads)
    torch.cuda.synchronize()
    V = len(cams)
    out = dict(
        feat=G.np_(rz.feat[: V * P]).copy(), radius=G.np_(rz.radius[: V * P]).copy(),
        tiles=G.np_(rz.tiles[: V * P]).copy(), depth=G.np_(rz.depth[: V * P]).copy(),
        gid=G.np_(rz.gid[: fr.M]).view(np.uint32).copy(), ranges=G.np_(rz.ranges[: rz.n_tiles]).view(np.uint32).copy(),
        img=G.np_(fr.flat_img).copy(), T=G.np_(fr.flat_T).copy(), last=G.np_(fr.flat_last).copy(),
        grad2d=G.np_(rz.grad2d[: V * P]).copy(), grads=G.np_(grads[:, :P]).copy(), M=fr.M)
    return out


def _tile_grid(cams, tile):
    """(view, tx, ty, W, H) of every global tile id, views in order."""
    out = []
    for v, c in enumerate(cams):
        W, H = c["width"], c["height"]
        TX, TY = -(-W // tile), -(-H // tile)
        for ty in range(TY):
            for tx in range(TX):
                out.append((v, tx, ty, W, H))
    return out


def _max_alpha_fp64(rec, px, py):
    """Largest alpha of the FP64 record (u, v, A, B, C, o) over pixel centres."""
    u, v, A, B, C, o = rec[:6]
    dx = px[None, :] - u
    dy = py[:, None] - v
    power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
    a = np.where(power <= 0.0, o * np.exp(np.minimum(power, 0.0)), 0.0)
    return float(a.max())


def _same_sums(a, b, scale_tol=1e-5):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.abs(b).max(axis=0, keepdims=True)
    err = np.abs(a - b)
    bad = err > 1e-4 * np.abs(b) + scale_tol * scale + 1e-12
    assert not bad.any(), (int(bad.sum()), float((err / (scale + 1e-30)).max()))


def _check(g, cams, tile, record=0, min_drop=0.0, mip2d=0.0, bg=(0.0, 0.0, 0.0), param_tol=1e-5):
    P = g.shape[0]
    V = len(cams)
    t = _run(g, cams, tile, 1, record, mip2d=mip2d, bg=bg)
    p = _run(g, cams, tile, 0, record, mip2d=mip2d, bg=bg)
    # projection: identical but for the mask words and the count
    np.testing.assert_array_equal(t["radius"], p["radius"])
    np.testing.assert_array_equal(t["depth"].view(np.uint32), p["depth"].view(np.uint32))
    ft, fp = t["feat"].reshape(-1, 12), p["feat"].reshape(-1, 12)
    np.testing.assert_array_equal(ft[:, :9].view(np.uint32), fp[:, :9].view(np.uint32))
    assert np.all(fp[:, 9:].view(np.uint32) == 0)
    assert np.all(t["tiles"] <= p["tiles"])
    masks = ft[:, 9].view(np.uint32).astype(np.uint64) | (ft[:, 10].view(np.uint32).astype(np.uint64) << np.uint64(32))
    has = masks != 0
    cnt = np.array([bin(int(m)).count("1") for m in masks])
    np.testing.assert_array_equal(t["tiles"][has], cnt[has])
    np.testing.assert_array_equal(t["tiles"][~has & (t["tiles"] > 0)], p["tiles"][~has & (t["tiles"] > 0)])
    assert t["M"] == int(t["tiles"].sum()) and p["M"] == int(p["tiles"].sum())
    assert t["M"] <= (1.0 - min_drop) * p["M"], (t["M"], p["M"])
    # the oracle's FP64 records of the same float32 parameters
    k = oracle.consts(tile=tile, sh_degree=3, mip2d=mip2d)
    o_feat = [oracle.project(G.f32(g), G.oracle_camera(c), k)["feat"] for c in cams]
    grid = _tile_grid(cams, tile)
    off = np.arange(tile) + 0.5
    dropped = 0
    for tid, (v, tx, ty, W, H) in enumerate(grid):
        a0, a1 = p["ranges"][tid]
        b0, b1 = t["ranges"][tid]
        lp = p["gid"][a0:a1]
        lt = t["gid"][b0:b1]
        if len(lt):
            at = {int(x): q for q, x in enumerate(lp)}
            order = np.array([at.get(int(x), -1) for x in lt])
            assert np.all(order >= 0), f"tile {tid}: tight entry not in the rect list"
            assert np.all(np.diff(order) > 0), f"tile {tid}: tight list out of order"
        gone = np.setdiff1d(lp, lt)
        if len(gone) == 0:
            continue
        px = tx * tile + off
        py = ty * tile + off
        px = px[px < W]
        py = py[py < H]
        for r in gone:
            dropped += 1
            i = int(r) - v * P
            amax = _max_alpha_fp64(o_feat[v][i], px, py)
            assert amax < ALPHA_MIN, f"tile {tid}: left out Gaussian {i} reaches alpha {amax}"
    assert dropped == p["M"] - t["M"]
    # compositing: same images and transmittances, same last blended Gaussian
    np.testing.assert_array_equal(t["img"].view(np.uint32), p["img"].view(np.uint32))
    np.testing.assert_array_equal(t["T"].view(np.uint32), p["T"].view(np.uint32))
    pix_tile = []
    for v, c in enumerate(cams):
        W, H = c["width"], c["height"]
        TX = -(-W // tile)
        base = sum(-(-cc["width"] // tile) * -(-cc["height"] // tile) for cc in cams[:v])
        yy, xx = np.mgrid[0:H, 0:W]
        pix_tile.append((base + (yy // tile) * TX + xx // tile).reshape(-1))
    pix_tile = np.concatenate(pix_tile)
    lt_, lp_ = t["last"].astype(np.int64), p["last"].astype(np.int64)
    np.testing.assert_array_equal(lt_ > 0, lp_ > 0)
    sel = lp_ > 0
    gl_t = t["gid"][t["ranges"][pix_tile[sel], 0].astype(np.int64) + lt_[sel] - 1]
    gl_p = p["gid"][p["ranges"][pix_tile[sel], 0].astype(np.int64) + lp_[sel] - 1]
    np.testing.assert_array_equal(gl_t, gl_p)
    # gradients: the same nonzero terms summed in another order by float
    # atomics; where terms cancel, the reordering error scales with the
    # column's magnitudes, so the absolute part is 1e-5 of the column's largest
    _same_sums(t["grad2d"].reshape(-1, 12)[:, :9], p["grad2d"].reshape(-1, 12)[:, :9])
    _same_sums(t["grads"].T, p["grads"].T, param_tol)
    return t["M"], p["M"]


@pytest.mark.parametrize("tile", [16, 8])
def test_cfg0_tight_lists(tile):
    g, cam, _ = U.cfg0_scene()
    _check(g, [cam], tile)


@pytest.fixture(scope="module")
def textured():
    g = synth.textured_scene(60_000, 1011)
    cams = synth.ring_cameras(8, 309, 205, 5.0, 2011)
    return g, cams


@pytest.mark.parametrize("tile,record", [(8, 0), (8, 1), (16, 0)])
def test_textured_tight_lists(textured, tile, record):
    g, cams = textured
    mt, mp = _check(g, [cams[0]], tile, record, min_drop=0.1)
    assert mt < mp


def test_textured_tight_lists_two_views(textured):
    g, cams = textured
    _check(g, [cams[1], cams[5]], 8, 0, min_drop=0.1)


def test_textured_tight_lists_mip_filter_and_background(textured):
    """The 2D filter scales each record's opacity (the mask's threshold follows
    it); a background colour changes no list."""
    g, cams = textured
    _check(g, [cams[2]], 8, 0, min_drop=0.1, mip2d=0.1, bg=(0.2, 0.5, 0.9))


@pytest.mark.parametrize("tile", [8, 16])
def test_needle_gaussians_tight_lists(tile):
    """Needle-like Gaussians (one long axis, two below the 2D dilation) at random
    orientations and opacities from just above 1/255: the projected ellipses
    reach elongations of several hundred to one, where the mask's margins are
    tightest; every left-out entry still stays below alpha 1/255 in FP64 and
    the images are the same bits.  The parameter gradients get a looser bound
    than the 2D ones: the projection's adjoint multiplies the 2D gradients'
    summation-order differences by the conditioning of these ellipses (their
    elongation, up to ~800 here)."""
    rng = np.random.default_rng(7)
    g = synth.random_gaussians(1500, 31)
    g[:, 3] = np.log(rng.uniform(0.05, 0.35, 1500))
    g[:, 4:6] = np.log(rng.uniform(0.001, 0.006, (1500, 2)))
    o = rng.uniform(0.005, 0.99, 1500)
    g[:, 10] = np.log(o / (1.0 - o))
    _check(g, [synth.camera_cfg0(160, 160, 4.0)], tile, min_drop=0.05, param_tol=5e-3)
