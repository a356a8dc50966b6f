"""End-to-end optimisation: plain full-resolution 3DGS training or DashGaussian's
scheduled training (resolution schedule + resolution-synced primitive budget),
with every step of every iteration in the CUDA library.

Per iteration k (Sec. 4; supplementary "Learning Rate", "Densification"):
  schedule step -> render size (H/r, W/r), position learning rate, P target;
  project -> bin -> render fwd -> L1 -> render bwd -> project bwd ->
  densification statistics -> Adam;
  every `densify_every` iterations in [densify_from, densify_until]: prune,
  Eq. 5 budget update with P_add = candidate count, Eq. 4 target, top-k
  clone/split (plain arm: every candidate, the 3DGS backbone);
  every `opacity_reset_every` iterations: opacity reset (3DGS backbone).
The plain arm renders every iteration at full resolution with the position
learning rate decaying from iteration 0.

Iterations count rendered views.  With V views per step (one multi-view
launch per pass, one Adam update per step), step j renders views jV .. jV+V-1
at the schedule's resolution for iteration jV, and the backbone's windows
(densification, opacity reset, learning-rate decay) stay in views seen; the
Adam hyper-parameters follow the batch-size rules of Grendel-GS (learning
rates x sqrt(V), betas^V, `dg_batch_adam_scale`).

Python here only orders the library calls and owns the device buffers
(PyTorch allocations); it computes nothing of the method.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time
from dataclasses import asdict, dataclass

import numpy as np
import torch

from . import capi
from .autotune import RenderTuner, Shape
from .graphstep import StepGraph
from .raster import Rasterizer, make_camera
from .schedule import spectrum_table


@dataclass
class TrainConfig:
    iters: int = 30000
    scheduled: bool = True
    # ablations of the scheduled arm (both on = the full method): resolution
    # schedule (render at floor(r(k)), position LR held until full resolution)
    # and primitive schedule (Eq. 4/5 budget, densification until full resolution)
    reso_sched: bool = True
    prim_sched: bool = True
    densify_from: int = 500
    densify_until: int = 15000
    densify_every: int = 100
    opacity_reset_every: int = 3000
    grad_thresh: float = 2e-4
    min_opacity: float = 0.005
    percent_dense: float = 0.01
    extent: float = 5.5
    P_cap: int = 3_000_000
    a: float = 4.0
    gamma: float = 0.98
    eta: float = 1.0
    lr_pos_init: float = 1.6e-4
    lr_pos_final: float = 1.6e-6
    lr_dc: float = 0.0025
    lr_rest: float = 0.0025 / 20
    lr_opacity: float = 0.025
    lr_scale: float = 0.005
    lr_rot: float = 0.001
    # 3DGS prunes "big points" (screen radius > 20 px, scale > 0.1 extent) after
    # the first opacity reset; off by default here because the synthetic ground
    # truth's Gaussians already have ~30 px radii at full resolution
    big_point_prune: bool = False
    # scheduled arm: keep densifying until the first full-resolution iteration
    # (Eq. 4 reaches P_fin there), so that the primitive growth curve spans the
    # optimisation as the paper describes, instead of stopping at densify_until
    densify_until_full: bool = True
    # backbone loss (1 - lambda) L1 + lambda D-SSIM; 0 trains on L1 alone
    ssim_lambda: float = 0.2
    # render launch shape: chosen per (image size, P) bucket by timing, or fixed
    autotune: bool = True
    # views rendered per step (one multi-view launch per pass) and capture of
    # the whole step in a CUDA graph (replayed with new cameras / LR / targets)
    views_per_step: int = 1
    cuda_graph: bool = False
    # records read by the render passes: 0 float32, 1 mixed (float16 conic and
    # opacity, bfloat16 colour; float32 transmittance, sums and gradients)
    record: int = 0
    # Sparse Adam (the Taming-3DGS backbone's optimiser): only Gaussians visible
    # in the step's views are updated
    sparse_adam: bool = False
    # Mip-Splatting's 2D filter in place of the dilation (backbone variant); 0 = off
    mip2d: float = 0.0
    # projection adjoint fused with the Adam update (no stored gradient, params
    # read once): 0.65 ms against 0.70 ms for the two kernels at 2M Gaussians;
    # sparse Adam always runs as its own kernel
    fused_adam: bool = True
    # V > 1: Adam learning rates x sqrt(V) and betas ^ V (Grendel-GS batch rules)
    batch_adam_scaling: bool = True
    # pair lists hold only the tiles where a Gaussian can reach alpha 1/255
    # (same images and gradients, shorter lists to sort and stage)
    tight_bins: bool = True
    seed: int = 0


class Trainer:
    def __init__(self, cfg: TrainConfig, init: np.ndarray, train_views, train_imgs, device="cuda"):
        """init: (P0, 59) parameters; train_views: camera dicts (full
        resolution); train_imgs: list of (3, H, W) float32 device tensors."""
        self.cfg = cfg
        self.dev = torch.device(device)
        self.views = train_views
        self.imgs = train_imgs
        self.H, self.W = train_imgs[0].shape[1], train_imgs[0].shape[2]
        # row stride a multiple of 4 floats: 16-byte row accesses in the Adam sweeps
        cap = (max(cfg.P_cap, init.shape[0]) + 1024 + 3) // 4 * 4
        self.cap = cap
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.buf = [dict(p=torch.zeros((59, cap), **f32), m=torch.zeros((59, cap), **f32),
                         v=torch.zeros((59, cap), **f32)) for _ in range(2)]
        self.cur = 0
        self.P = init.shape[0]
        self.buf[0]["p"][:, : self.P] = torch.from_numpy(np.ascontiguousarray(init.T.astype(np.float32))).to(self.dev)
        self.grads = torch.zeros((59, cap), **f32)
        self.acc = torch.zeros(cap, **f32)
        self.den = torch.zeros(cap, **f32)
        self.maxr = torch.zeros(cap, **f32)
        self.tuner = RenderTuner(self.dev, capi.raster_opts(record=cfg.record, mip2d=cfg.mip2d, tight_bins=int(cfg.tight_bins)),
                                 fixed=None if cfg.autotune else Shape(16, 2, 4, 0))
        self.rz = self.tuner.rasterizer(Shape(8, 1, 1, 0))  # evaluation renders
        n_full = 3 * self.H * self.W
        self.dL = torch.empty(n_full, **f32)
        self.loss = torch.zeros(2, **f32)
        self.lws = torch.empty(capi.dg_loss_workspace_size(n_full), dtype=torch.uint8, device=self.dev)
        self.sws = torch.empty(capi.dg_ssim_workspace_size([(self.W, self.H)]), dtype=torch.uint8, device=self.dev)
        self.dws = None
        self.counts = torch.zeros(2, dtype=torch.int64, device=self.dev)
        self.P_out = torch.zeros(1, dtype=torch.int64, device=self.dev)
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(cfg.seed)
        self.order_rng = np.random.default_rng(cfg.seed)
        self.order = []
        self.gt_cache = {}
        self.stream = torch.cuda.current_stream(self.dev)
        self.sched = None
        self.V = max(1, cfg.views_per_step)
        self.n_steps = (cfg.iters + self.V - 1) // self.V
        self.beta1, self.beta2 = 0.9, 0.999
        if self.V > 1 and cfg.batch_adam_scaling:
            _, self.beta1, self.beta2 = capi.dg_batch_adam_scale(self.V, [0.0] * 59, 0.9, 0.999)
        # the iteration plan (render size, position LR) of the plain arm; the
        # scheduled arm replaces it with the resolution schedule in init_schedule
        self.plan_sched = capi.dg_schedule_init_plain(self.H, self.W, self._sched_params())
        self._full_cams = {}
        self.history = []
        self.init_schedule_s = 0.0
        self.densify_until = cfg.densify_until
        self.graphs = {}
        self._cam_cache = {}
        self.graph_P = -1
        self.M_hint = {}
        self.pending = []  # replayed steps whose status is still to be read
        self.skipped_steps = 0
        self.graph_captures = 0
        self.capture_s = 0.0  # host seconds in graph captures (each also runs its step)
        self.densify_s = 0.0  # host seconds in densification (two host reads of device counts)

    # ---------------------------------------------------------------- schedule
    def _sched_params(self):
        cfg = self.cfg
        return capi.sched_params(cfg.iters, a=cfg.a, gamma=cfg.gamma, eta=cfg.eta, P_init=float(self.P),
                                 P_cap=float(cfg.P_cap), lr_pos_init=cfg.lr_pos_init * cfg.extent,
                                 lr_pos_final=cfg.lr_pos_final * cfg.extent)

    def init_schedule(self):
        t0 = time.perf_counter()
        cfg = self.cfg
        _, sat = spectrum_table(self.imgs, self.dev)
        self.sched = capi.dg_schedule_init(sat, self.H, self.W, self._sched_params())
        if cfg.reso_sched:
            self.plan_sched = self.sched
        if cfg.densify_until_full and cfg.prim_sched:
            self.densify_until = max(cfg.densify_until, int(self.sched.k_full))
        torch.cuda.synchronize()
        self.init_schedule_s = time.perf_counter() - t0

    def _plan(self, it):
        """(r_mod, h, w, position LR) at iteration `it` (views rendered so far)."""
        o = capi.dg_schedule_step(self.plan_sched, it)
        return o.r_mod, o.height, o.width, o.lr_pos

    def _target(self, j, r, h, w):
        if r == 1:
            return self.imgs[j]
        key = (j, r)
        t = self.gt_cache.get(key)
        if t is None:
            t = torch.empty((3, h, w), dtype=torch.float32, device=self.dev)
            capi.dg_downsample_area(self.imgs[j], 3, self.H, self.W, t, h, w, self.stream)
            self.gt_cache[key] = t
        return t

    def _camera(self, j, h, w):
        key = (j, h, w)
        c = self._cam_cache.get(key)
        if c is None:
            full = self._full_cams.get(j)
            if full is None:
                v = self.views[j]
                full = make_camera(np.asarray(v["viewmat"], np.float32).reshape(-1), v["intr"], self.W, self.H)
                self._full_cams[j] = full
            c = capi.dg_camera_scale(full, w, h)
            self._cam_cache[key] = c
        return c

    def _next_view(self):
        if not self.order:
            self.order = list(self.order_rng.permutation(len(self.views)))
        return int(self.order.pop())

    # ---------------------------------------------------------------- step
    def _lr(self, lr_pos):
        cfg = self.cfg
        lr = [lr_pos] * 3 + [cfg.lr_scale] * 3 + [cfg.lr_rot] * 4 + [cfg.lr_opacity] + [cfg.lr_dc] * 3 + \
            [cfg.lr_rest] * 45
        if self.V > 1 and cfg.batch_adam_scaling:
            lr, _, _ = capi.dg_batch_adam_scale(self.V, lr, 0.9, 0.999)
        return lr

    def _step_batched(self, k):
        """V views per step through the multi-view calls; with cuda_graph the
        whole step is one graph replay."""
        cfg = self.cfg
        b = self.buf[self.cur]
        P = self.P
        V = self.V
        it = k * V
        r, h, w, lr_pos = self._plan(it)
        js = [self._next_view() for _ in range(V)]
        cams = [self._camera(j, h, w) for j in js]
        targets = [self._target(j, r, h, w) for j in js]
        lr = self._lr(lr_pos)
        b1, b2 = self.beta1, self.beta2
        stats_on = it < self.densify_until
        if not cfg.cuda_graph:
            shape, rz, key = self.tuner.pick(V * h * w, P)
            e0 = self.tuner.start(self.stream)
            params = b["p"][:, :P]
            fr = rz.forward(params, P, cams, self.stream)
            tgt = torch.cat([t.reshape(-1) for t in targets])
            n = tgt.numel()
            capi.dg_loss_l1_dssim(fr.flat_img, tgt, [(w, h)] * V, cfg.ssim_lambda, self.dL_b(n), self.loss_b(V),
                                  self.sws_b([(w, h)] * V), self.sws_batch.numel(), self.stream)
            rz.backward_render(fr, self._dLb[:n], self.stream)
            self.tuner.stop(key, shape, e0, self.stream)
            if stats_on:
                capi.dg_densify_stats(rz.grad2d, rz.radius, P, cams, V, self.acc, self.den, self.maxr, self.stream)
            if cfg.fused_adam and not cfg.sparse_adam:
                capi.dg_project_bwd_adam(b["p"], self.cap, P, cams, V, rz.opts, rz.radius, rz.clamp, rz.grad2d,
                                         None, b["m"], b["v"], lr, b1, b2, 1e-15, k + 1, self.stream)
            else:
                capi.dg_project_bwd(params, self.cap, P, cams, V, rz.opts, rz.radius, rz.clamp, rz.grad2d,
                                    self.grads[:, :P], self.stream)
                self._adam(b, P, lr, k, rz.radius, V)
            return r, fr.M
        # graph path: one graph per (P, size, stats window, buffer set); the
        # status of a step is read two steps later, so the host prepares the
        # next step while the GPU runs the current one
        self._check_pending(keep=1)
        if P != self.graph_P:
            self.graphs.clear()
            self.graph_P = P
        hp = capi.dg_adam_hparams_fill(lr, b1, b2, 1e-15, k + 1)
        key = (P, h, w, V, stats_on, self.cur)
        g = self.graphs.get(key)
        if g is None:
            hint = self.M_hint.get((w, h))
            if hint is None:  # first batch at this size: count its pairs once
                rz0 = self.tuner.rasterizer(Shape(8, 1, 1, 0))
                fr0 = rz0.forward(b["p"][:, :P], P, cams, self.stream)
                hint = fr0.M
            M_cap = int(hint * 1.5) + 4096
            g = StepGraph(self.dev, capi.raster_opts(tile=8, record=cfg.record, mip2d=cfg.mip2d,
                                                   tight_bins=int(cfg.tight_bins)), 1, 1, b["p"],
                          b["m"], b["v"],
                          self.grads, self.cap, P,
                          cams, M_cap, cfg.ssim_lambda, (self.acc, self.den, self.maxr) if stats_on else None,
                          fused=cfg.fused_adam)
            g.key = key
            tc = time.perf_counter()
            slot = g.capture(cams, hp, targets)
            self.capture_s += time.perf_counter() - tc
            self.graphs[key] = g
            self.graph_captures += 1
        else:
            slot = g.replay(cams, hp, targets)
        self.pending.append((g, slot))
        self.loss = g.loss
        return r, -1

    def _check_pending(self, keep):
        """Reads the status of all but the last `keep` replayed steps."""
        while len(self.pending) > keep:
            g_prev, slot = self.pending.pop(0)
            status, M = g_prev.result(slot)
            sz = g_prev.sizes[0]
            self.M_hint[sz] = max(self.M_hint.get(sz, 0), M)
            if status != 0:  # pair capacity exceeded: that step made no update
                self.skipped_steps += 1
                self.graphs.pop(g_prev.key, None)

    def _adam(self, b, P, lr, k, radius, V):
        if self.cfg.sparse_adam:
            if getattr(self, "vis", None) is None or self.vis.numel() < self.cap:
                self.vis = torch.zeros(self.cap, dtype=torch.uint8, device=self.dev)
            capi.dg_visibility(radius, P, V, self.vis, self.stream)
            capi.dg_sparse_adam_step(b["p"], self.grads, b["m"], b["v"], self.cap, P, lr, self.beta1, self.beta2,
                                     1e-15, k + 1, self.vis, self.stream)
        else:
            capi.dg_adam_step(b["p"], self.grads, b["m"], b["v"], self.cap, P, lr, self.beta1, self.beta2, 1e-15,
                              k + 1, self.stream)

    def dL_b(self, n):
        if getattr(self, "_dLb", None) is None or self._dLb.numel() < n:
            self._dLb = torch.empty(n, dtype=torch.float32, device=self.dev)
        return self._dLb

    def loss_b(self, V):
        if self.loss.numel() < V + 1:
            self.loss = torch.zeros(V + 1, dtype=torch.float32, device=self.dev)
        return self.loss

    def sws_b(self, sizes):
        need = capi.dg_ssim_workspace_size(sizes)
        if getattr(self, "sws_batch", None) is None or self.sws_batch.numel() < need:
            self.sws_batch = torch.empty(need, dtype=torch.uint8, device=self.dev)
        return self.sws_batch

    def step(self, k):
        """Step k: views kV .. kV+V-1.  The backbone's events (densification,
        opacity reset) fire when their iteration falls inside the step."""
        cfg = self.cfg
        if self.V > 1 or cfg.cuda_graph:
            r, M = self._step_batched(k)
        else:
            r, M = self._step_single(k)
        it0, it1 = k * self.V, (k + 1) * self.V
        kk = it1 // cfg.densify_every * cfg.densify_every
        if kk > it0 and cfg.densify_from <= kk <= self.densify_until:
            self.densify(kk)
        kk = it1 // cfg.opacity_reset_every * cfg.opacity_reset_every
        if kk > it0 and kk <= cfg.densify_until:
            b = self.buf[self.cur]
            capi.dg_opacity_reset(b["p"], b["m"], b["v"], self.cap, self.P, 0.01, self.stream)
        return r, M

    def _step_single(self, k):
        cfg = self.cfg
        b = self.buf[self.cur]
        P = self.P
        r, h, w, lr_pos = self._plan(k)
        j = self._next_view()
        cam = self._camera(j, h, w)
        params = b["p"][:, :P]
        shape, rz, key = self.tuner.pick(h * w, P)
        e0 = self.tuner.start(self.stream)
        fr = rz.forward(params, P, cam, self.stream)
        n = 3 * h * w
        tgt = self._target(j, r, h, w)
        if cfg.ssim_lambda > 0:
            capi.dg_loss_l1_dssim(fr.img, tgt, [(w, h)], cfg.ssim_lambda, self.dL, self.loss, self.sws,
                                  self.sws.numel(), self.stream)
        else:
            capi.dg_loss_l1(fr.img, tgt, n, self.dL, self.loss, self.lws, self.lws.numel(), self.stream)
        rz.backward_render(fr, self.dL[:n].view(3, h, w), self.stream)
        self.tuner.stop(key, shape, e0, self.stream)
        if k < self.densify_until:
            capi.dg_densify_stats(rz.grad2d, rz.radius, P, cam, 1, self.acc, self.den, self.maxr, self.stream)
        lr = self._lr(lr_pos)
        if cfg.fused_adam and not cfg.sparse_adam:
            rz.project_bwd_adam(b["p"], self.cap, fr, b["m"], b["v"], lr, k + 1, stream=self.stream)
        else:
            capi.dg_project_bwd(params, self.cap, P, cam, 1, rz.opts, rz.radius, rz.clamp, rz.grad2d,
                                self.grads[:, :P], self.stream)
            self._adam(b, P, lr, k, rz.radius, 1)
        return r, fr.M

    def densify(self, k):
        td = time.perf_counter()
        self._densify(k)
        self.densify_s += time.perf_counter() - td

    def _densify(self, k):
        cfg = self.cfg
        P = self.P
        b = self.buf[self.cur]
        dst = self.buf[1 - self.cur]
        need = capi.dg_densify_workspace_size(P)
        if self.dws is None or self.dws.numel() < need:
            self.dws = torch.empty(int(need * 1.2) + 1024, dtype=torch.uint8, device=self.dev)
        big = cfg.big_point_prune and k > cfg.opacity_reset_every
        # the loss of a V-view step is the mean over its views, so each view's
        # screen-space gradient carries a factor 1/V: the per-view threshold
        # scales with it
        opts = capi.densify_opts(cfg.grad_thresh / cfg.views_per_step, cfg.min_opacity, cfg.percent_dense,
                                 cfg.extent, 20.0 if big else 0.0, 0.1 * cfg.extent if big else 0.0)
        capi.dg_densify_mark(b["p"], self.cap, P, self.acc, self.den, self.maxr, opts, self.dws, self.dws.numel(),
                             self.counts, self.stream)
        n_keep, n_cand = (int(x) for x in self.counts.cpu())
        # Eq. 5 / Eq. 4 budget (primitive schedule) or every candidate (backbone), capped
        sched = self.sched if (self.sched is not None and cfg.prim_sched) else None
        budget, _ = capi.dg_densify_budget(sched, k, n_keep, n_cand, cfg.P_cap)
        n_sel = min(budget, n_cand)
        noise = torch.randn((max(n_sel, 1), 2, 3), generator=self.gen, device=self.dev)
        capi.dg_densify_apply(b["p"], b["m"], b["v"], self.cap, P, n_cand, budget, noise, self.dws, self.dws.numel(),
                              dst["p"], dst["m"], dst["v"], self.cap, self.P_out, self.stream)
        self.P = int(self.P_out.item())
        self.cur = 1 - self.cur
        self.acc.zero_(); self.den.zero_(); self.maxr.zero_()
        self.history.append(dict(iter=k, P=self.P, n_keep=n_keep, n_cand=n_cand, budget=budget))

    # ---------------------------------------------------------------- eval
    def psnr(self, views, imgs):
        b = self.buf[self.cur]
        out = torch.zeros(1, dtype=torch.float32, device=self.dev)
        vals = []
        for v, gt in zip(views, imgs):
            cam = make_camera(np.asarray(v["viewmat"], np.float32).reshape(-1), v["intr"], self.W, self.H)
            fr = self.rz.forward(b["p"][:, : self.P], self.P, cam, self.stream)
            capi.dg_mse(fr.img, gt, 3 * self.H * self.W, out, self.lws, self.lws.numel(), self.stream)
            vals.append(-10.0 * math.log10(max(float(out.item()), 1e-12)))
        return float(np.mean(vals))

    def run(self, log_every=0):
        cfg = self.cfg
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if cfg.scheduled:
            self.init_schedule()
        res_hist = {}
        for k in range(self.n_steps):
            r, M = self.step(k)
            res_hist[r] = res_hist.get(r, 0) + self.V
            if log_every and ((k + 1) * self.V) % log_every < self.V:
                torch.cuda.synchronize()
                print(json.dumps(dict(iter=(k + 1) * self.V, P=self.P, r=r, loss=float(self.loss[0].item()),
                                      s=round(time.perf_counter() - t0, 2))), flush=True)
        torch.cuda.synchronize()
        self._check_pending(keep=0)
        return dict(seconds=time.perf_counter() - t0, schedule_init_s=self.init_schedule_s, P_final=self.P,
                    iters_per_factor={str(k): v for k, v in sorted(res_hist.items())},
                    render_shapes=self.tuner.summary(), views_per_step=self.V, steps=self.n_steps,
                    cuda_graph=cfg.cuda_graph, graph_captures=self.graph_captures,
                    skipped_steps=self.skipped_steps, densify_events=len(self.history),
                    host_densify_s=round(self.densify_s, 3), host_capture_s=round(self.capture_s, 3))


def make_dataset(n_gt, n_views, W, H, device, seed=1001, gt=None):
    """GT scene (generated, or the given one), cameras and GT renders; every
    8th view held out."""
    from . import synth
    if gt is None:
        gt = synth.textured_scene(n_gt, seed)
    cams = synth.ring_cameras(n_views, W, H, 5.0, seed + 1000)
    rz = Rasterizer(device, capi.raster_opts())
    gtp = torch.from_numpy(np.ascontiguousarray(gt.T)).to(device)
    imgs = []
    for v in cams:
        cam = make_camera(np.asarray(v["viewmat"], np.float32).reshape(-1), v["intr"], W, H)
        imgs.append(rz.forward(gtp, gt.shape[0], cam).img.clone())
    del gtp
    test = [i for i in range(n_views) if i % 8 == 0]
    train = [i for i in range(n_views) if i % 8 != 0]
    return gt, cams, imgs, train, test


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--arm", choices=["plain", "scheduled", "both", "reso", "prim", "all"], default="both",
                    help="both = plain + scheduled; reso / prim = the scheduled arm with only the resolution / "
                         "only the primitive schedule; all = the four")
    ap.add_argument("--a", type=float, default=4.0, help="r_m from X(r_m) = X(1)/a (Sec. 4.2)")
    ap.add_argument("--gamma", type=float, default=0.98, help="Eq. 5 momentum")
    ap.add_argument("--iters", type=int, default=30000, help="views rendered (steps x views per step)")
    ap.add_argument("--n-gt", type=int, default=2_000_000)
    ap.add_argument("--seed", type=int, default=1001,
                    help="scene seed (cameras seed + 1000); 1000 + k for configuration k")
    ap.add_argument("--n-init", type=int, default=100_000)
    ap.add_argument("--views", type=int, default=160)
    ap.add_argument("--width", type=int, default=1237)
    ap.add_argument("--height", type=int, default=822)
    ap.add_argument("--p-cap", type=int, default=3_000_000)
    ap.add_argument("--log-every", type=int, default=0)
    ap.add_argument("--ssim-lambda", type=float, default=0.2)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--views-per-step", type=int, default=1)
    ap.add_argument("--cuda-graph", action="store_true", help="capture each step in a CUDA graph")
    ap.add_argument("--sparse-adam", action="store_true", help="update only visible Gaussians (Taming-3DGS)")
    ap.add_argument("--mip2d", type=float, default=0.0, help="Mip-Splatting 2D filter variance (0: dilation)")
    ap.add_argument("--record", choices=["fp32", "mixed"], default="fp32",
                    help="render-side record storage (mixed: float16 conic/opacity, bfloat16 colour)")
    ap.add_argument("--runs", nargs="*", default=None,
                    help="several runs on one dataset, each 'arm[:key=value...]' with keys a, gamma, v (views per "
                         "step), graph (0/1), record (fp32/mixed), sparse (0/1), mip2d, iters; e.g. plain "
                         "scheduled:a=4:v=16:graph=1:record=mixed (default: the runs --arm names)")
    args = ap.parse_args(argv)
    from . import synth
    dev = torch.device("cuda")
    gt, cams, imgs, train, test = make_dataset(args.n_gt, args.views, args.width, args.height, dev, seed=args.seed)
    init = synth.perturb(gt, 3001, n_keep=args.n_init)
    runs = args.runs or {"both": ["plain", "scheduled"],
                         "all": ["plain", "scheduled", "reso", "prim"]}.get(args.arm, [args.arm])
    results = {}
    for spec in runs:
        res, _ = train_run(spec, args, init, cams, imgs, train, test, dev)
        results[spec] = res
        print(json.dumps({spec: res}), flush=True)
    print(json.dumps(dict(config=vars(args), results=results)), flush=True)
    return results


def parse_run(spec: str, args) -> TrainConfig:
    """TrainConfig of one run spec 'arm[:key=value...]' (defaults from args)."""
    parts = spec.split(":")
    arm = parts[0]
    if arm not in ("plain", "scheduled", "reso", "prim"):
        raise ValueError(f"unknown arm {arm!r} in {spec!r}")
    kv = dict(p.split("=", 1) for p in parts[1:])
    iters = int(kv.pop("iters", args.iters))
    cfg = TrainConfig(iters=iters, scheduled=(arm != "plain"), P_cap=args.p_cap,
                      reso_sched=arm in ("scheduled", "reso"), prim_sched=arm in ("scheduled", "prim"),
                      a=float(kv.pop("a", args.a)), gamma=float(kv.pop("gamma", args.gamma)),
                      ssim_lambda=args.ssim_lambda, autotune=not args.no_autotune,
                      views_per_step=int(kv.pop("v", args.views_per_step)),
                      cuda_graph=bool(int(kv.pop("graph", int(args.cuda_graph)))),
                      record=1 if kv.pop("record", args.record) == "mixed" else 0,
                      sparse_adam=bool(int(kv.pop("sparse", int(args.sparse_adam)))),
                      mip2d=float(kv.pop("mip2d", args.mip2d)))
    if kv:
        raise ValueError(f"unknown keys {sorted(kv)} in {spec!r}")
    if iters < 30000:  # compress the backbone's iteration windows proportionally
        s = iters / 30000
        cfg.densify_from = max(1, int(500 * s)); cfg.densify_until = int(15000 * s)
        cfg.densify_every = max(1, int(100 * s)); cfg.opacity_reset_every = max(1, int(3000 * s))
    return cfg


def train_run(spec, args, init, cams, imgs, train, test, dev):
    """One training run; returns (result dict, its TrainConfig)."""
    cfg = parse_run(spec, args)
    tr = Trainer(cfg, init, [cams[i] for i in train], [imgs[i] for i in train], dev)
    res = tr.run(log_every=args.log_every)
    res["psnr_test"] = tr.psnr([cams[i] for i in test], [imgs[i] for i in test])
    res["densify_last"] = tr.history[-1] if tr.history else None
    if tr.sched is not None:
        s = tr.sched
        res["schedule"] = dict(r_m=s.r_m, m=s.m, k_full=s.k_full, P_fin=s.P_fin,
                               anchors=[(s.s[i], s.r[i]) for i in range(s.m + 1)])
    del tr
    torch.cuda.empty_cache()
    return res, cfg


if __name__ == "__main__":
    sys.exit(0 if main() else 1)
