"""Python glue around the C ABI: buffer management and torch.autograd.

``Rasterizer`` owns the device buffers of one view (projected records,
binning workspace, pair list, per-pixel state) and grows them on demand;
every step of the computation runs in the CUDA library through ``capi``.
``rasterize`` is the differentiable entry point: a ``torch.autograd.Function``
whose backward calls dg_render_bwd and dg_project_bwd.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import capi

NPARAM = capi.NPARAM


def make_camera(viewmat, intr, width, height) -> capi.Camera:
    fx, fy, cx, cy = intr
    return capi.camera(viewmat, fx, fy, cx, cy, width, height)


@dataclass
class Frame:
    """Per-view forward state kept for the backward pass."""
    P: int
    cam: capi.Camera
    img: torch.Tensor       # (3, H, W)
    T: torch.Tensor         # (H, W)
    last: torch.Tensor      # (H, W) int32
    M: int                  # number of (tile, Gaussian) pairs


class Rasterizer:
    """Reusable buffers for rendering P Gaussians into one view at a time."""

    def __init__(self, device="cuda", opts: capi.RasterOpts | None = None, pair_headroom: float = 1.25,
                 ppt_fwd: int | None = None, ppt_bwd: int | None = None):
        self.device = torch.device(device)
        self.opts = opts if opts is not None else capi.raster_opts()
        # launch shape of each render pass (pixels per thread); None keeps opts'
        self.opts_fwd = self._with_ppt(self.opts, ppt_fwd)
        self.opts_bwd = self._with_ppt(self.opts, ppt_bwd)
        self.headroom = pair_headroom
        self.P_cap = -1
        self.M_cap = 0
        self.n_tiles = 0
        self.ws = None
        self.examined = None
        self.mark = None  # optional callback(stage_name) after each stage, for event timing

    @staticmethod
    def _with_ppt(opts, ppt):
        o = capi.RasterOpts.from_buffer_copy(opts)
        if ppt is not None:
            o.pixels_per_thread = int(ppt)
        return o

    def _mark(self, name):
        if self.mark is not None:
            self.mark(name)

    # ------------------------------------------------------------ buffers
    def _ensure_prims(self, P):
        if P <= self.P_cap:
            return
        d = self.device
        n = max(P, 1)
        self.feat = torch.empty((n, capi.FEAT_FLOATS), dtype=torch.float32, device=d)
        self.depth = torch.empty(n, dtype=torch.float32, device=d)
        self.radius = torch.empty(n, dtype=torch.int32, device=d)
        self.tiles = torch.empty(n, dtype=torch.int32, device=d)
        self.clamp = torch.empty(n, dtype=torch.uint8, device=d)
        self.grad2d = torch.empty((n, capi.FEAT_FLOATS), dtype=torch.float32, device=d)
        self.M_dev = torch.zeros(1, dtype=torch.int64, device=d)
        self.status = torch.zeros(1, dtype=torch.int32, device=d)
        self.P_cap = P
        self.ws = None

    def _ensure_ws(self, P, M_cap, n_tiles):
        need = capi.dg_bin_workspace_size(P, M_cap, n_tiles)
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        if M_cap > self.M_cap or not hasattr(self, "gid"):
            self.gid = torch.empty(max(M_cap, 1), dtype=torch.int32, device=self.device)
            self.M_cap = M_cap

    def _ensure_tiles(self, n_tiles):
        if n_tiles > self.n_tiles:
            self.ranges = torch.empty((n_tiles, 2), dtype=torch.int32, device=self.device)
            self.n_tiles = n_tiles

    # ------------------------------------------------------------ passes
    def forward(self, params: torch.Tensor, P: int, cam: capi.Camera, stream=None,
                examined: bool = False) -> Frame:
        """Project, bin, sort and composite P Gaussians of the planar
        [59, stride] float32 tensor ``params`` into view ``cam``."""
        assert params.dtype == torch.float32 and params.shape[0] == NPARAM and params.stride(1) == 1
        stream = stream or torch.cuda.current_stream(self.device)
        B = self.opts.tile
        W, H = cam.width, cam.height
        n_tiles = ((W + B - 1) // B) * ((H + B - 1) // B)
        self._ensure_prims(P)
        self._ensure_tiles(n_tiles)
        stride = params.stride(0)
        capi.dg_project(params, stride, P, cam, self.opts, self.feat, self.depth, self.radius, self.tiles,
                        self.clamp, stream)
        self._mark("project")
        self._ensure_ws(P, max(self.M_cap, 1), n_tiles)
        capi.dg_bin_count(self.depth, self.tiles, P, self.ws, self.ws.numel(), self.M_cap, n_tiles,
                          self.M_dev, stream)
        self._mark("bin_count")
        stream.synchronize()
        M = int(self.M_dev.item())
        if M > self.M_cap:
            self._ensure_ws(P, int(M * self.headroom) + 1024, n_tiles)
            capi.dg_bin_count(self.depth, self.tiles, P, self.ws, self.ws.numel(), self.M_cap, n_tiles,
                              self.M_dev, stream)
        self._mark("host_sync")
        capi.dg_bin_sort(self.feat, self.radius, P, cam, B, self.ws, self.ws.numel(), self.M_cap, self.gid,
                         self.ranges, self.status, stream)
        self._mark("bin_sort")
        img = torch.empty((3, H, W), dtype=torch.float32, device=self.device)
        T = torch.empty((H, W), dtype=torch.float32, device=self.device)
        last = torch.empty((H, W), dtype=torch.int32, device=self.device)
        ex = bl = None
        if examined:
            ex = torch.empty((H, W), dtype=torch.int32, device=self.device)
            bl = torch.empty((H, W), dtype=torch.int32, device=self.device)
            self.examined = ex
            self.blended = bl
        capi.dg_render_fwd(self.feat, self.gid, self.ranges, cam, self.opts_fwd, img, T, last, ex, bl, stream)
        self._mark("render_fwd")
        return Frame(P=P, cam=cam, img=img, T=T, last=last, M=M)

    def backward(self, params: torch.Tensor, fr: Frame, dL_dimg: torch.Tensor, grads: torch.Tensor,
                 stream=None) -> None:
        """Writes dL/dparams of the frame into the planar ``grads`` (same stride as params)."""
        stream = stream or torch.cuda.current_stream(self.device)
        assert dL_dimg.is_contiguous() and dL_dimg.dtype == torch.float32
        capi.dg_render_bwd(self.feat, self.gid, self.ranges, fr.cam, self.opts_bwd, fr.T, fr.last, dL_dimg, fr.P,
                           self.grad2d, stream)
        self._mark("render_bwd")
        capi.dg_project_bwd(params, params.stride(0), fr.P, fr.cam, self.opts, self.radius, self.clamp,
                            self.grad2d, grads, stream)
        self._mark("project_bwd")


class _RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, rasterizer, cam):
        fr = rasterizer.forward(params, params.shape[1], cam)
        ctx.rasterizer = rasterizer
        ctx.frame = fr
        ctx.save_for_backward(params)
        return fr.img

    @staticmethod
    def backward(ctx, dL_dimg):
        (params,) = ctx.saved_tensors
        grads = torch.empty_like(params)
        ctx.rasterizer.backward(params, ctx.frame, dL_dimg.contiguous(), grads)
        return grads, None, None


def rasterize(params: torch.Tensor, rasterizer: Rasterizer, cam: capi.Camera) -> torch.Tensor:
    """Differentiable render of the planar [59, P] float32 parameters into ``cam``.

    The backward recomputes each pixel's transmittance from the stored final
    T and last contributor and returns dL/dparams with the same layout.  The
    rasterizer's buffers hold the state of the most recent call, so call
    backward before rendering the next view with the same rasterizer."""
    return _RasterizeFn.apply(params, rasterizer, cam)
