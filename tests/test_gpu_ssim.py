"""CUDA L1 + D-SSIM loss vs the FP64 oracle (needs a GPU).

Tolerances, from the float32 arithmetic: the loss is a mean of per-pixel
terms each within ~1e-6 relative, accumulated per block in float32 and
across blocks in FP64: 1e-5 absolute.  The gradient of pixel q combines
three 121-term window sums of partial derivatives whose size is bounded by
1/(C1 C2)-scaled ratios of local statistics; on images in [0, 1] those
ratios stay O(10), so 1e-4 relative to the largest gradient entry holds
with margin (the per-pixel gradient is compared after multiplying by the
pixel count, its natural scale).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ssim as OS  # noqa: E402
from paper_2503_18402_gb300 import capi  # noqa: E402

pytestmark = pytest.mark.gpu


def _run(imgs, tgts, lam):
    sizes = [(x.shape[2], x.shape[1]) for x in imgs]
    img = torch.from_numpy(np.concatenate([x.reshape(-1) for x in imgs]).astype(np.float32)).cuda()
    tgt = torch.from_numpy(np.concatenate([x.reshape(-1) for x in tgts]).astype(np.float32)).cuda()
    dL = torch.empty_like(img)
    loss = torch.zeros(len(sizes) + 1, device="cuda")
    ws = torch.empty(capi.dg_ssim_workspace_size(sizes), dtype=torch.uint8, device="cuda")
    capi.dg_loss_l1_dssim(img, tgt, sizes, lam, dL, loss, ws, ws.numel())
    torch.cuda.synchronize()
    out, off = [], 0
    g = dL.cpu().numpy()
    for (W, H) in sizes:
        out.append(g[off: off + 3 * W * H].reshape(3, H, W))
        off += 3 * W * H
    return loss.cpu().numpy(), out


def _check(imgs, tgts, lam=0.2):
    loss, grads = _run(imgs, tgts, lam)
    V = len(imgs)
    ref_losses = []
    for v in range(V):
        x = imgs[v].astype(np.float32).astype(np.float64)
        y = tgts[v].astype(np.float32).astype(np.float64)
        lv, gv = OS.l1_dssim(x, y, lam)
        ref_losses.append(lv)
        assert abs(loss[v] - lv) <= 1e-5, (v, loss[v], lv)
        # gradient of the mean over views, at the per-pixel scale
        n = x.size * V
        got, ref = grads[v].astype(np.float64) * n, gv * x.size
        # L1 ties (x == y) are exact zeros on both sides; compare everything
        err = np.abs(got - ref)
        assert err.max() <= 1e-4 * np.abs(ref).max() + 1e-6, (v, err.max(), np.abs(ref).max())
    assert abs(loss[V] - np.mean(ref_losses)) <= 1e-5


@pytest.mark.parametrize("W,H", [(64, 64), (130, 99), (37, 5), (1, 1), (33, 70)])
def test_single_view_matches_oracle(W, H):
    rng = np.random.default_rng(W * 1000 + H)
    x = rng.random((3, H, W))
    y = np.clip(x + 0.2 * rng.normal(size=x.shape), 0, 1)
    _check([x], [y])


def test_views_of_uneven_sizes_in_one_call():
    rng = np.random.default_rng(7)
    sizes = [(64, 48), (97, 31), (20, 20)]
    xs = [rng.random((3, H, W)) for W, H in sizes]
    ys = [rng.random((3, H, W)) for W, H in sizes]
    _check(xs, ys, lam=0.2)
    _check(xs, ys, lam=0.7)


def test_identical_images_and_lambda_zero():
    rng = np.random.default_rng(8)
    x = rng.random((3, 40, 50))
    loss, g = _run([x], [x], 0.2)
    assert abs(loss[0]) <= 1e-6  # L1 = 0 and SSIM = 1
    assert np.abs(g[0]).max() <= 1e-6 / x.size * 10
    # lambda = 0 is the L1 loss of dg_loss_l1, gradient bit for bit
    y = rng.random((3, 40, 50))
    loss0, g0 = _run([x], [y], 0.0)
    img = torch.from_numpy(x.astype(np.float32).reshape(-1)).cuda()
    tgt = torch.from_numpy(y.astype(np.float32).reshape(-1)).cuda()
    dL = torch.empty_like(img)
    l1 = torch.zeros(1, device="cuda")
    ws = torch.empty(capi.dg_loss_workspace_size(img.numel()), dtype=torch.uint8, device="cuda")
    capi.dg_loss_l1(img, tgt, img.numel(), dL, l1, ws, ws.numel())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g0[0].reshape(-1), dL.cpu().numpy())
    assert abs(loss0[0] - l1.item()) <= 1e-6


def test_full_resolution_sampled():
    """1237 x 822 render-sized images: loss vs the oracle's full evaluation."""
    rng = np.random.default_rng(9)
    W, H = 1237, 822
    x = rng.random((3, H, W)).astype(np.float32)
    # a smooth target (large SSIM variance range), not white noise
    yy, xx = np.mgrid[0:H, 0:W]
    y = np.stack([0.5 + 0.4 * np.sin(xx / (17.0 + 5 * c) + yy / 23.0) for c in range(3)]).astype(np.float32)
    _check([x], [y])


def test_argument_errors():
    t = torch.zeros(3 * 8 * 8, device="cuda")
    with pytest.raises(capi.DashGSError):
        capi.dg_loss_l1_dssim(t, t, [(8, 8)], 1.5, t, t, t, 0)
    assert capi.dg_ssim_workspace_size([(0, 8)]) == 0
    with pytest.raises(capi.DashGSError) as e:
        capi.dg_loss_l1_dssim(t, t, [(8, 8)], 0.2, t, t, torch.zeros(16, dtype=torch.uint8, device="cuda"), 16)
    assert "workspace" in str(e.value)
