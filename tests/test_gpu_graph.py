"""Graph-replayable forms of the step (needs a GPU): cameras and Adam
hyper-parameters read from device memory give the same bits as the host
forms; the Adam skip flag holds the update; a captured step replays the
direct sequence; a short batched training run with graph capture learns."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_18402_gb300 import capi, synth  # noqa: E402
from paper_2503_18402_gb300.graphstep import StepGraph  # noqa: E402
from paper_2503_18402_gb300.raster import Rasterizer  # noqa: E402
from tests import _gpu as G  # noqa: E402

pytestmark = pytest.mark.gpu


def _cams_dev(cams):
    arr = capi.cameras(cams)
    raw = np.frombuffer(ctypes.string_at(ctypes.addressof(arr), ctypes.sizeof(arr)), dtype=np.uint8)
    return torch.from_numpy(raw.copy()).cuda()


def _scene(n=4000, seed=3):
    g = synth.random_gaussians(n, seed)
    g[:, 3:6] += 0.3
    sizes = [(64, 64), (90, 50), (40, 70)]
    cams = [G.gpu_camera(synth.camera_cfg0(W, H, 4.0 + 0.6 * i)) for i, (W, H) in enumerate(sizes)]
    return g, cams


def test_device_cameras_give_the_host_bits():
    g, cams = _scene()
    P, V = g.shape[0], len(cams)
    params = G.gpu_params(g)
    opts = capi.raster_opts()
    outs = []
    for dev in (None, _cams_dev(cams)):
        feat = torch.zeros((V * P, 12), device="cuda")
        depth = torch.zeros(V * P, device="cuda")
        radius = torch.zeros(V * P, dtype=torch.int32, device="cuda")
        tiles = torch.zeros(V * P, dtype=torch.int32, device="cuda")
        clamp = torch.zeros(V * P, dtype=torch.uint8, device="cuda")
        capi.dg_project(params, params.stride(0), P, cams, V, opts, feat, depth, radius, tiles, clamp, cams_dev=dev)
        g2 = torch.from_numpy(np.random.default_rng(0).normal(size=(V * P, 12)).astype(np.float32) * 1e-3).cuda()
        grads = torch.zeros_like(params)
        capi.dg_project_bwd(params, params.stride(0), P, cams, V, opts, radius, clamp, g2, grads, cams_dev=dev)
        torch.cuda.synchronize()
        outs.append([G.np_(x) for x in (feat, depth, radius, tiles, clamp, grads)])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


def test_adam_from_device_hparams_and_skip_flag():
    rng = np.random.default_rng(1)
    P, stride = 1003, 1010
    p0 = rng.normal(size=(59, stride)).astype(np.float32)
    gr = torch.from_numpy(rng.normal(size=(59, stride)).astype(np.float32)).cuda()
    lr = np.linspace(1e-4, 1e-2, 59).astype(np.float32)
    a = [torch.from_numpy(p0.copy()).cuda(), torch.zeros((59, stride), device="cuda"), torch.zeros((59, stride), device="cuda")]
    capi.dg_adam_step(a[0], gr, a[1], a[2], stride, P, lr, 0.9, 0.999, 1e-15, 5)
    hp = capi.dg_adam_hparams_fill(lr, 0.9, 0.999, 1e-15, 5)
    raw = np.frombuffer(ctypes.string_at(ctypes.addressof(hp), ctypes.sizeof(hp)), dtype=np.uint8).copy()
    hp_dev = torch.from_numpy(raw).cuda()
    b = [torch.from_numpy(p0.copy()).cuda(), torch.zeros((59, stride), device="cuda"), torch.zeros((59, stride), device="cuda")]
    zero = torch.zeros(1, dtype=torch.int32, device="cuda")
    capi.dg_adam_step_dev(b[0], gr, b[1], b[2], stride, P, hp_dev, skip_if=zero)
    c = [torch.from_numpy(p0.copy()).cuda(), torch.zeros((59, stride), device="cuda"), torch.zeros((59, stride), device="cuda")]
    capi.dg_adam_step_dev(c[0], gr, c[1], c[2], stride, P, hp_dev, skip_if=torch.full((1,), -2, dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(G.np_(x), G.np_(y))
    np.testing.assert_array_equal(G.np_(c[0]), p0)  # skipped: untouched
    assert float(c[1].abs().max()) == 0.0


@pytest.mark.parametrize("fused", [False, True])
def test_captured_step_replays_the_direct_sequence(fused):
    """The captured step (projection adjoint and Adam as two kernels, or
    fused) equals the direct sequence of calls.  Fused, the gradient is not
    stored; it is read from the first moment, which after step 1 from zero
    moments is (1 - beta1) g."""
    g, cams = _scene(3000, 5)
    P, V = g.shape[0], len(cams)
    stride = P + 7
    base = np.zeros((59, stride), np.float32)
    base[:, :P] = g.T
    rng = np.random.default_rng(2)
    targets = [torch.from_numpy(rng.random((3, c.height, c.width)).astype(np.float32)).cuda() for c in cams]
    lr = [1e-4] * 59
    # direct sequence
    params = torch.from_numpy(base.copy()).cuda()
    m, v, grads = torch.zeros_like(params), torch.zeros_like(params), torch.zeros_like(params)
    rz = Rasterizer("cuda", capi.raster_opts(tile=8))
    fr = rz.forward(params[:, :P], P, cams)
    tgt = torch.cat([t.reshape(-1) for t in targets])
    dL = torch.empty_like(tgt)
    loss = torch.zeros(V + 1, device="cuda")
    sizes = [(c.width, c.height) for c in cams]
    sws = torch.empty(capi.dg_ssim_workspace_size(sizes), dtype=torch.uint8, device="cuda")
    capi.dg_loss_l1_dssim(fr.flat_img, tgt, sizes, 0.2, dL, loss, sws, sws.numel())
    rz.backward_render(fr, dL)
    capi.dg_project_bwd(params[:, :P], stride, P, cams, V, rz.opts, rz.radius, rz.clamp, rz.grad2d, grads[:, :P])
    capi.dg_adam_step(params, grads, m, v, stride, P, lr, 0.9, 0.999, 1e-15, 1)
    torch.cuda.synchronize()
    img_direct = G.np_(fr.flat_img).copy()
    # captured: the capture's warm-up performs step 1, a replay then step 2 on
    # the same inputs from the same start
    params2 = torch.from_numpy(base.copy()).cuda()
    m2, v2, grads2 = torch.zeros_like(params2), torch.zeros_like(params2), torch.zeros_like(params2)
    sg = StepGraph("cuda", capi.raster_opts(tile=8), 1, 1, params2, m2, v2, grads2, stride, P, cams, fr.M + 100, 0.2,
                   fused=fused)

    def step_grad():
        return G.np_(m2[:, :P]) / np.float32(0.1) if fused else G.np_(grads2[:, :P])
    hp1 = capi.dg_adam_hparams_fill(lr, 0.9, 0.999, 1e-15, 1)
    sg.capture(cams, hp1, targets)
    status, M = sg.result()
    assert status == 0 and M == fr.M
    np.testing.assert_array_equal(G.np_(sg.rz.fixed["img"]), img_direct)
    np.testing.assert_allclose(G.np_(sg.loss), G.np_(loss), rtol=0, atol=1e-7)
    ok, worst, nbad = G.grad_close(step_grad(), G.np_(grads[:, :P]))
    assert ok, (worst, nbad)
    # replay with the step-1 state restored: same result again
    params2.copy_(torch.from_numpy(base.copy()).cuda()); m2.zero_(); v2.zero_()
    sg.replay(cams, hp1, targets)
    status, M = sg.result()
    assert status == 0
    np.testing.assert_array_equal(G.np_(sg.rz.fixed["img"]), img_direct)
    ok, worst, nbad = G.grad_close(step_grad(), G.np_(grads[:, :P]))
    assert ok, (worst, nbad)
    # new cameras through the same graph: equals a direct render of them
    cams_b = [G.gpu_camera(synth.camera_cfg0(c.width, c.height, 3.5 + 0.4 * i)) for i, c in enumerate(cams)]
    params2.copy_(torch.from_numpy(base.copy()).cuda()); m2.zero_(); v2.zero_()
    sg.replay(cams_b, hp1, targets)
    status, M = sg.result()
    fr_b = Rasterizer("cuda", capi.raster_opts(tile=8)).forward(torch.from_numpy(base.copy()).cuda()[:, :P], P, cams_b)
    torch.cuda.synchronize()
    if M <= sg.M_cap:
        assert status == 0
        np.testing.assert_array_equal(G.np_(sg.rz.fixed["img"]), G.np_(fr_b.flat_img))
    else:  # capacity exceeded: reported, and Adam held the update
        assert status != 0
        np.testing.assert_array_equal(G.np_(params2), base)


def test_batched_graph_training_learns():
    from paper_2503_18402_gb300.train import Trainer, TrainConfig, make_dataset
    dev = torch.device("cuda")
    gt, cams, imgs, train, test = make_dataset(40_000, 16, 160, 106, dev)
    init = synth.perturb(gt, 3001, n_keep=4000)
    cfg = TrainConfig(iters=300, views_per_step=4, cuda_graph=True, densify_from=30, densify_until=200,
                      densify_every=30, opacity_reset_every=300, P_cap=20_000)
    tr = Trainer(cfg, init, [cams[i] for i in train], [imgs[i] for i in train])
    tv, ti = [cams[i] for i in test], [imgs[i] for i in test]
    psnr0 = tr.psnr(tv, ti)
    res = tr.run()
    psnr1 = tr.psnr(tv, ti)
    assert psnr1 > psnr0 + 2.0, (psnr0, psnr1)
    assert res["graph_captures"] >= 1 and res["skipped_steps"] <= 2
