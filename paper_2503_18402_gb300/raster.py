"""Python glue around the C ABI: buffer management and torch.autograd.

``Rasterizer`` owns the device buffers of one batch of views (projected
records, binning workspace, pair list, per-pixel state) and grows them on
demand; every step of the computation runs in the CUDA library through
``capi``.  ``rasterize`` is the differentiable entry point: a
``torch.autograd.Function`` whose backward calls dg_render_bwd and
dg_project_bwd.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import capi

NPARAM = capi.NPARAM


def make_camera(viewmat, intr, width, height) -> capi.Camera:
    fx, fy, cx, cy = intr
    return capi.camera(viewmat, fx, fy, cx, cy, width, height)


@dataclass
class Frame:
    """Forward state of one batch of views, kept for the backward pass.
    With one view, img/T/last are shaped (3, H, W)/(H, W)/(H, W); with several
    they are the flat concatenations and `images`, `Ts`, `lasts` hold the
    per-view slices."""
    P: int
    cams: list
    img: torch.Tensor
    T: torch.Tensor
    last: torch.Tensor
    M: int
    flat_img: torch.Tensor = None
    flat_T: torch.Tensor = None
    flat_last: torch.Tensor = None
    images: list = field(default_factory=list)
    Ts: list = field(default_factory=list)
    lasts: list = field(default_factory=list)


class Rasterizer:
    """Reusable buffers for rendering P Gaussians into one or more views."""

    def __init__(self, device="cuda", opts: capi.RasterOpts | None = None, pair_headroom: float = 1.25,
                 ppt_fwd: int | None = None, ppt_bwd: int | None = None):
        self.device = torch.device(device)
        self.opts = opts if opts is not None else capi.raster_opts()
        # launch shape of each render pass (pixels per thread); None keeps opts'
        self.opts_fwd = self._with_ppt(self.opts, ppt_fwd)
        self.opts_bwd = self._with_ppt(self.opts, ppt_bwd)
        self.headroom = pair_headroom
        self.N_cap = -1
        self.M_cap = 0
        self.n_tiles = 0
        self.ws = None
        self.rws = None  # render workspace, shared by a batch's forward and backward
        self.examined = None
        self.blended = None
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
    def _ensure_records(self, N):
        if N <= self.N_cap:
            return
        d = self.device
        n = max(N, 1)
        self.feat = torch.empty((n, capi.FEAT_FLOATS), dtype=torch.float32, device=d)
        self.depth = torch.empty(n, dtype=torch.float32, device=d)
        self.radius = torch.empty(n, dtype=torch.int32, device=d)
        self.tiles = torch.empty(n, dtype=torch.int32, device=d)
        self.clamp = torch.empty(n, dtype=torch.uint8, device=d)
        self.grad2d = torch.empty((n, capi.FEAT_FLOATS), dtype=torch.float32, device=d)
        # mixed-precision copy of the records read by the render passes (opts.record == 1)
        self.packed = (torch.empty(n * capi.PACKED_RECORD_BYTES, dtype=torch.uint8, device=d)
                       if self.opts.record == 1 else None)
        self.M_dev = torch.zeros(1, dtype=torch.int64, device=d)
        # pinned landing slot of the pair count: one async copy and one event wait
        self.M_host = torch.zeros(1, dtype=torch.int64).pin_memory()
        self.M_event = torch.cuda.Event()
        self.status = torch.zeros(1, dtype=torch.int32, device=d)
        self.N_cap = N
        self.ws = None

    def _ensure_ws(self, P, n_views, M_cap):
        need = capi.dg_bin_workspace_size(P, n_views, M_cap)
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        if M_cap > self.M_cap or not hasattr(self, "gid"):
            self.gid = torch.empty(max(M_cap, 1), dtype=torch.int32, device=self.device)
            self.M_cap = M_cap

    def _pack(self, n_records, stream):
        """Render-side records: the float32 ones, or their mixed-precision packing."""
        if self.opts.record == 1:
            capi.dg_pack_records(self.feat, n_records, self.packed, stream)
            return self.packed
        return self.feat

    def _ensure_tiles(self, n_tiles):
        if n_tiles > self.n_tiles:
            self.ranges = torch.empty((n_tiles, 2), dtype=torch.int32, device=self.device)
            self.n_tiles = n_tiles

    def _ensure_rws(self, carr, V):
        need = capi.dg_render_workspace_size(carr, V, self.opts_fwd, self.M_cap)
        if self.rws is None or self.rws.numel() < need:
            self.rws = torch.empty(need, dtype=torch.uint8, device=self.device)

    # ------------------------------------------------------------ fixed-capacity passes
    def prepare(self, P: int, cams, M_cap: int) -> None:
        """Allocates every buffer a batch of these cameras needs with room for
        M_cap pairs, so that forward_fixed/backward_render allocate nothing
        (as required inside a CUDA graph capture)."""
        cams = [cams] if isinstance(cams, capi.Camera) else list(cams)
        V = len(cams)
        carr = capi.cameras(cams)
        B = self.opts.tile
        n_tiles = sum(((c.width + B - 1) // B) * ((c.height + B - 1) // B) for c in cams)
        npix = sum(c.width * c.height for c in cams)
        self._ensure_records(V * P)
        self._ensure_tiles(n_tiles)
        self._ensure_ws(P, V, max(int(M_cap), self.M_cap, 1))
        self._ensure_rws(carr, V)
        d = self.device
        self.fixed = dict(img=torch.empty(3 * npix, dtype=torch.float32, device=d),
                          T=torch.empty(npix, dtype=torch.float32, device=d),
                          last=torch.empty(npix, dtype=torch.int32, device=d))

    def forward_fixed(self, params: torch.Tensor, P: int, cams, stream=None, cams_dev=None) -> Frame:
        """forward() without the host read of the pair count: bins with the
        capacity set by prepare() (a larger count sets the device status word
        self.status to DG_ERR_CAPACITY and renders empty tiles); no allocation,
        no synchronisation.  cams_dev: optional device copy of the cameras."""
        cams = [cams] if isinstance(cams, capi.Camera) else list(cams)
        V = len(cams)
        carr = capi.cameras(cams)
        stream = stream or torch.cuda.current_stream(self.device)
        B = self.opts.tile
        capi.dg_project(params, params.stride(0), P, carr, V, self.opts, self.feat, self.depth, self.radius,
                        self.tiles, self.clamp, stream, cams_dev=cams_dev)
        capi.dg_bin_count(self.depth, self.tiles, P, V, self.ws, self.ws.numel(), self.M_cap, self.M_dev, stream)
        capi.dg_bin_sort(self.feat, self.radius, P, carr, V, B, self.ws, self.ws.numel(), self.M_cap, self.gid,
                         self.ranges, self.status, stream)
        f = self.fixed
        self.rfeat = self._pack(V * P, stream)
        capi.dg_render_fwd(self.rfeat, self.gid, self.ranges, carr, V, self.opts_fwd, f["img"], f["T"], f["last"],
                           None, None, self.rws, self.rws.numel(), stream)
        return Frame(P=P, cams=cams, img=f["img"], T=f["T"], last=f["last"], M=-1, flat_img=f["img"],
                     flat_T=f["T"], flat_last=f["last"])

    # ------------------------------------------------------------ passes
    def forward(self, params: torch.Tensor, P: int, cams, stream=None, examined: bool = False) -> Frame:
        """Project, bin, sort and composite P Gaussians of the planar
        [59, stride] float32 tensor ``params`` into one camera or a list of
        cameras (at most 16)."""
        assert params.dtype == torch.float32 and params.shape[0] == NPARAM and params.stride(1) == 1
        cams = [cams] if isinstance(cams, capi.Camera) else list(cams)
        V = len(cams)
        carr = capi.cameras(cams)
        stream = stream or torch.cuda.current_stream(self.device)
        B = self.opts.tile
        sizes = [(c.width, c.height) for c in cams]
        n_tiles = sum(((W + B - 1) // B) * ((H + B - 1) // B) for W, H in sizes)
        npix = sum(W * H for W, H in sizes)
        self._ensure_records(V * P)
        self._ensure_tiles(n_tiles)
        stride = params.stride(0)
        capi.dg_project(params, stride, P, carr, V, self.opts, self.feat, self.depth, self.radius, self.tiles,
                        self.clamp, stream)
        self._mark("project")
        self._ensure_ws(P, V, max(self.M_cap, 1))
        capi.dg_bin_count(self.depth, self.tiles, P, V, self.ws, self.ws.numel(), self.M_cap, self.M_dev, stream)
        self._mark("bin_count")
        with torch.cuda.stream(stream):
            self.M_host.copy_(self.M_dev, non_blocking=True)
        self.M_event.record(stream)
        # the pair sort is queued before the count reaches the host, so the GPU
        # runs on while the host waits; when the pairs exceed the capacity it
        # only records DG_ERR_CAPACITY (nothing written) and is redone below
        capi.dg_bin_sort(self.feat, self.radius, P, carr, V, B, self.ws, self.ws.numel(), self.M_cap, self.gid,
                         self.ranges, self.status, stream)
        self._mark("bin_sort")
        self.M_event.synchronize()
        M = int(self.M_host[0])
        if M > self.M_cap:
            self._ensure_ws(P, V, int(M * self.headroom) + 1024)
            capi.dg_bin_count(self.depth, self.tiles, P, V, self.ws, self.ws.numel(), self.M_cap, self.M_dev, stream)
            capi.dg_bin_sort(self.feat, self.radius, P, carr, V, B, self.ws, self.ws.numel(), self.M_cap, self.gid,
                             self.ranges, self.status, stream)
        self._mark("host_sync")
        img = torch.empty(3 * npix, dtype=torch.float32, device=self.device)
        T = torch.empty(npix, dtype=torch.float32, device=self.device)
        last = torch.empty(npix, dtype=torch.int32, device=self.device)
        ex = bl = None
        if examined:
            ex = torch.empty(npix, dtype=torch.int32, device=self.device)
            bl = torch.empty(npix, dtype=torch.int32, device=self.device)
        self._ensure_rws(carr, V)
        self.rfeat = self._pack(V * P, stream)
        capi.dg_render_fwd(self.rfeat, self.gid, self.ranges, carr, V, self.opts_fwd, img, T, last, ex, bl,
                           self.rws, self.rws.numel(), stream)
        self._mark("render_fwd")
        fr = Frame(P=P, cams=cams, img=img, T=T, last=last, M=M, flat_img=img, flat_T=T, flat_last=last)
        off = 0
        exs, bls = [], []
        for W, H in sizes:
            fr.images.append(img[3 * off: 3 * (off + W * H)].view(3, H, W))
            fr.Ts.append(T[off: off + W * H].view(H, W))
            fr.lasts.append(last[off: off + W * H].view(H, W))
            if examined:
                exs.append(ex[off: off + W * H].view(H, W))
                bls.append(bl[off: off + W * H].view(H, W))
            off += W * H
        if V == 1:
            fr.img, fr.T, fr.last = fr.images[0], fr.Ts[0], fr.lasts[0]
        if examined:
            self.examined = exs[0] if V == 1 else exs
            self.blended = bls[0] if V == 1 else bls
        return fr

    def backward_render(self, fr: Frame, dL_dimg: torch.Tensor, stream=None) -> None:
        """Render adjoint only: fills self.grad2d (per-record 2D gradients)."""
        stream = stream or torch.cuda.current_stream(self.device)
        assert dL_dimg.is_contiguous() and dL_dimg.dtype == torch.float32
        assert dL_dimg.numel() == fr.flat_img.numel()
        carr = capi.cameras(fr.cams)
        V = len(fr.cams)
        capi.dg_render_bwd(self.rfeat, self.gid, self.ranges, carr, V, self.opts_bwd, fr.flat_T, fr.flat_last,
                           dL_dimg, V * fr.P, self.grad2d, self.rws, self.rws.numel(), stream)
        self._mark("render_bwd")

    def project_bwd_adam(self, params: torch.Tensor, stride: int, fr: Frame, m, v, lr, step, beta1=0.9,
                         beta2=0.999, eps=1e-15, grads=None, stream=None) -> None:
        """Projection adjoint fused with the Adam update of params/m/v
        (planar [59][stride] buffers holding at least fr.P Gaussians)."""
        stream = stream or torch.cuda.current_stream(self.device)
        carr = capi.cameras(fr.cams)
        capi.dg_project_bwd_adam(params, stride, fr.P, carr, len(fr.cams), self.opts, self.radius, self.clamp,
                                 self.grad2d, grads, m, v, lr, beta1, beta2, eps, step, stream)
        self._mark("project_bwd_adam")

    def backward(self, params: torch.Tensor, fr: Frame, dL_dimg: torch.Tensor, grads: torch.Tensor,
                 stream=None) -> None:
        """Writes dL/dparams of the frame (summed over its views) into the
        planar ``grads`` (same stride as params).  dL_dimg: the frame's image
        layout ((3, H, W) for one view, the flat concatenation otherwise)."""
        stream = stream or torch.cuda.current_stream(self.device)
        assert dL_dimg.is_contiguous() and dL_dimg.dtype == torch.float32
        assert dL_dimg.numel() == fr.flat_img.numel()
        carr = capi.cameras(fr.cams)
        V = len(fr.cams)
        capi.dg_render_bwd(self.rfeat, self.gid, self.ranges, carr, V, self.opts_bwd, fr.flat_T, fr.flat_last,
                           dL_dimg, V * fr.P, self.grad2d, self.rws, self.rws.numel(), stream)
        self._mark("render_bwd")
        capi.dg_project_bwd(params, params.stride(0), fr.P, carr, V, self.opts, self.radius, self.clamp,
                            self.grad2d, grads, stream)
        self._mark("project_bwd")


class _RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, rasterizer, cams):
        fr = rasterizer.forward(params, params.shape[1], cams)
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


def rasterize(params: torch.Tensor, rasterizer: Rasterizer, cams) -> torch.Tensor:
    """Differentiable render of the planar [59, P] float32 parameters into one
    camera ((3, H, W) output) or a list of cameras (flat concatenation).

    The backward recomputes each pixel's transmittance from the stored final
    T and last contributor and returns dL/dparams with the same layout.  The
    rasterizer's buffers hold the state of the most recent call, so call
    backward before rendering the next batch with the same rasterizer."""
    return _RasterizeFn.apply(params, rasterizer, cams)
