"""Python glue for the schedule entry points (buffers only; the arithmetic is
in the CUDA library and its host-side C++ schedule)."""
from __future__ import annotations

import torch

from . import capi


def spectrum_table(views, device="cuda", stream=None):
    """Runs dg_spectrum_accumulate over the training views ((3, H, W) float32
    tensors on the device) and dg_spectrum_finalize.  Returns the DC-centred
    view-mean spectrum (device, float64) and its summed-area table (host numpy)."""
    views = list(views)
    H, W = views[0].shape[1], views[0].shape[2]
    stream = stream or torch.cuda.current_stream(device)
    acc = torch.zeros((H, W), dtype=torch.float64, device=device)
    ws = torch.empty(capi.dg_spectrum_workspace_size(H, W), dtype=torch.uint8, device=device)
    for v in views:
        assert v.shape == (3, H, W) and v.dtype == torch.float32 and v.is_contiguous()
        capi.dg_spectrum_accumulate(v, H, W, acc, ws, ws.numel(), stream)
    shifted = torch.empty((H, W), dtype=torch.float64, device=device)
    sat = torch.empty((H + 1, W + 1), dtype=torch.float64, device=device)
    capi.dg_spectrum_finalize(acc, len(views), H, W, shifted, sat, stream)
    return shifted, sat.cpu().numpy()


def build_schedule(views, S, **params):
    """Spectrum of the training views -> dg_schedule (host struct)."""
    shifted, sat = spectrum_table(views)
    H, W = shifted.shape
    return capi.dg_schedule_init(sat, H, W, capi.sched_params(S, **params))


def downsample(img: torch.Tensor, h: int, w: int, stream=None) -> torch.Tensor:
    C, H, W = img.shape
    out = torch.empty((C, h, w), dtype=torch.float32, device=img.device)
    capi.dg_downsample_area(img.contiguous(), C, H, W, out, h, w, stream or torch.cuda.current_stream(img.device))
    return out
