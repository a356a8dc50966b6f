"""One training step of V views captured as a CUDA graph and replayed.

The step is the whole per-iteration path -- projection, binning, forward,
L1 + D-SSIM loss, backward, densification statistics, projection adjoint and
Adam -- as one graph, so an iteration costs one graph launch instead of
dozens of kernel launches and the host never waits on the GPU inside it.

What changes between replays lives in device buffers the kernels read when
they run: the cameras (``cams_dev``, read by the projection and its adjoint),
the Adam hyper-parameters (``hp_dev``: position learning rate and step
count), and the targets (copied into the graph's target buffer before the
launch).  What is fixed in a graph: the Gaussian count P, the image sizes,
the launch shape and the pair capacity M_cap.  The projection adjoint and
Adam run as one kernel (dg_project_bwd_adam_dev) unless ``fused`` is off.
The binning writes a device status word when a step needs more than M_cap
pairs; Adam then skips its update (the skip flag), and the caller, which reads the status
and the pair count asynchronously after the replay, re-captures with a
larger capacity and repeats the step.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi
from .raster import Rasterizer


class StepGraph:
    def __init__(self, device, opts: capi.RasterOpts, ppt_fwd, ppt_bwd, params, m, v, grads, stride: int, P: int,
                 cams, M_cap: int, ssim_lambda: float, stats=None, fused: bool = True):
        """params/m/v/grads: planar [59][stride] buffers (fixed addresses;
        grads is unused when fused); cams: host cameras of the batch (their
        sizes fix the graph); stats: (acc, den, maxr) densification
        accumulators, or None."""
        self.device = torch.device(device)
        self.P = P
        self.V = len(cams)
        self.sizes = [(c.width, c.height) for c in cams]
        self.cams = list(cams)
        self.M_cap = int(M_cap)
        self.rz = Rasterizer(self.device, opts, ppt_fwd=ppt_fwd, ppt_bwd=ppt_bwd)
        self.rz.prepare(P, self.cams, self.M_cap)
        d = self.device
        npix = sum(w * h for w, h in self.sizes)
        self.target = torch.empty(3 * npix, dtype=torch.float32, device=d)
        self.dL = torch.empty(3 * npix, dtype=torch.float32, device=d)
        self.loss = torch.zeros(self.V + 1, dtype=torch.float32, device=d)
        self.sws = torch.empty(capi.dg_ssim_workspace_size(self.sizes), dtype=torch.uint8, device=d)
        cam_bytes = ctypes.sizeof(capi.Camera) * self.V
        hp_bytes = ctypes.sizeof(capi.AdamHparams)
        self.cams_dev = torch.empty(cam_bytes, dtype=torch.uint8, device=d)
        self.hp_dev = torch.empty(hp_bytes, dtype=torch.uint8, device=d)
        # two pinned staging slots: the host fills one while the copies of the
        # previous step may still read the other
        self.cams_host = [torch.empty(cam_bytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
        self.hp_host = [torch.empty(hp_bytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
        self.slot_event = [torch.cuda.Event(), torch.cuda.Event()]
        self.slot = 0
        # per staging slot: (status, pair count) of the step that used the slot
        self.out_host = [torch.zeros(2, dtype=torch.int64).pin_memory() for _ in range(2)]
        self.out_event = [torch.cuda.Event(), torch.cuda.Event()]
        self.status64 = torch.zeros(1, dtype=torch.int64, device=d)
        self.params, self.m, self.v, self.grads, self.stride = params, m, v, grads, stride
        self.lam = ssim_lambda
        self.stats = stats
        self.fused = fused
        self.graph = None

    def _sequence(self, stream):
        rz = self.rz
        carr = capi.cameras(self.cams)
        prm = self.params[:, : self.P]
        fr = rz.forward_fixed(prm, self.P, self.cams, stream, cams_dev=self.cams_dev)
        capi.dg_loss_l1_dssim(fr.img, self.target, self.sizes, self.lam, self.dL, self.loss, self.sws,
                              self.sws.numel(), stream)
        rz.backward_render(fr, self.dL, stream)
        if self.stats is not None:
            acc, den, maxr = self.stats
            capi.dg_densify_stats(rz.grad2d, rz.radius, self.P, carr, self.V, acc, den, maxr, stream)
        if self.fused:
            capi.dg_project_bwd_adam_dev(self.params, self.stride, self.P, carr, self.V, rz.opts, rz.radius, rz.clamp,
                                         rz.grad2d, None, self.m, self.v, self.hp_dev, skip_if=rz.status,
                                         stream=stream, cams_dev=self.cams_dev)
            return
        capi.dg_project_bwd(prm, self.stride, self.P, carr, self.V, rz.opts, rz.radius, rz.clamp, rz.grad2d,
                            self.grads[:, : self.P], stream, cams_dev=self.cams_dev)
        capi.dg_adam_step_dev(self.params, self.grads, self.m, self.v, self.stride, self.P, self.hp_dev,
                              skip_if=rz.status, stream=stream)

    def _write_inputs(self, cams, hp: capi.AdamHparams, targets, stream) -> int:
        k = self.slot
        self.slot = 1 - k
        self.slot_event[k].synchronize()  # the copies that last read this slot are done
        csz = ctypes.sizeof(capi.Camera)
        base = self.cams_host[k].data_ptr()
        for v, c in enumerate(cams):
            ctypes.memmove(base + v * csz, ctypes.addressof(c), csz)
        ctypes.memmove(self.hp_host[k].data_ptr(), ctypes.addressof(hp), ctypes.sizeof(hp))
        with torch.cuda.stream(stream):
            self.cams_dev.copy_(self.cams_host[k], non_blocking=True)
            self.hp_dev.copy_(self.hp_host[k], non_blocking=True)
            self.slot_event[k].record(stream)
            off = 0
            for t in targets:
                n = t.numel()
                self.target[off: off + n].copy_(t.reshape(-1), non_blocking=True)
                off += n
        return k

    def capture(self, cams, hp, targets) -> int:
        """Warm-up run (which also performs a step), then capture.  Returns the
        slot holding that step's result (see result())."""
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        k = self._write_inputs(cams, hp, targets, s)
        with torch.cuda.stream(s):
            self._sequence(s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        self._finish(torch.cuda.current_stream(self.device), k)
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize(self.device)
        with torch.cuda.graph(g, stream=s):
            self._sequence(s)
        self.graph = g
        return k

    def replay(self, cams, hp, targets) -> int:
        stream = torch.cuda.current_stream(self.device)
        k = self._write_inputs(cams, hp, targets, stream)
        self.graph.replay()
        self._finish(stream, k)
        return k

    def _finish(self, stream, k):
        with torch.cuda.stream(stream):
            self.status64.copy_(self.rz.status)
            self.out_host[k][0:1].copy_(self.status64, non_blocking=True)
            self.out_host[k][1:2].copy_(self.rz.M_dev, non_blocking=True)
        self.out_event[k].record(stream)

    def result(self, k=None):
        """(status, pair count) of the step that used slot k (default: the
        latest); waits for that step."""
        if k is None:
            k = 1 - self.slot
        self.out_event[k].synchronize()
        return int(self.out_host[k][0]), int(self.out_host[k][1])
