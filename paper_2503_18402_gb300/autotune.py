"""Launch-shape autotuner for the render passes.

Every candidate shape computes the same image and gradients (up to float
rounding order); they differ in speed, and which one is fastest depends on
the image size and the Gaussian count: small images have few tiles with long
lists (list splitting pays), large ones have many tiles (splitting costs its
extra product pass, smaller tiles cut wasted evaluations).  The tuner times
the forward + backward of real training iterations with CUDA events,
cycling through the candidates for each (pixel-count, Gaussian-count)
bucket, then keeps the fastest for that bucket.  Events are read only once
they have completed (no synchronisation is added to the loop).

A shape is (tile edge, pixels per thread of the forward and the backward
pass, list splitting: -1 never, 0 automatic).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import capi
from .raster import Rasterizer


@dataclass(frozen=True)
class Shape:
    tile: int
    ppt_fwd: int
    ppt_bwd: int
    split: int

    def label(self) -> str:
        return f"t{self.tile}f{self.ppt_fwd}b{self.ppt_bwd}s{self.split}"


CANDIDATES = (
    Shape(8, 1, 1, 0),
    Shape(8, 1, 1, -1),
    Shape(8, 2, 2, 0),
    Shape(8, 1, 2, 0),
    Shape(16, 2, 4, 0),
    Shape(16, 1, 1, 0),
    Shape(16, 2, 2, -1),
)


def bucket(npix: int, P: int) -> tuple:
    """Half-octave buckets of the pixel count and octaves of P."""
    return (int(round(2 * math.log2(max(npix, 1)))), max(int(P), 1).bit_length())


class RenderTuner:
    def __init__(self, device="cuda", opts: capi.RasterOpts | None = None, candidates=CANDIDATES,
                 trials: int = 2, fixed: Shape | None = None):
        self.device = torch.device(device)
        self.base = opts if opts is not None else capi.raster_opts()
        self.candidates = tuple(candidates)
        self.trials = trials
        self.fixed = fixed
        self.rz = {}
        self.best = {}
        self.times = {}
        self.pending = []

    def rasterizer(self, shape: Shape) -> Rasterizer:
        r = self.rz.get(shape)
        if r is None:
            o = capi.RasterOpts.from_buffer_copy(self.base)
            o.tile = shape.tile
            o.split_len = shape.split
            r = Rasterizer(self.device, o, ppt_fwd=shape.ppt_fwd, ppt_bwd=shape.ppt_bwd)
            self.rz[shape] = r
        return r

    def _drain(self):
        keep = []
        for key, shape, e0, e1 in self.pending:
            if e1.query():
                self.times.setdefault(key, {}).setdefault(shape, []).append(e0.elapsed_time(e1))
            else:
                keep.append((key, shape, e0, e1))
        self.pending = keep
        for key, per in self.times.items():
            if key in self.best:
                continue
            # the first timing of each shape is a warm-up (buffer growth, first launch)
            if all(len(per.get(s, ())) >= self.trials + 1 for s in self.candidates):
                self.best[key] = min(self.candidates, key=lambda s: sorted(per[s][1:])[len(per[s][1:]) // 2])

    def pick(self, npix: int, P: int):
        """Shape and rasterizer for the next iteration; returns (shape, rasterizer, key)."""
        if self.fixed is not None:
            return self.fixed, self.rasterizer(self.fixed), None
        self._drain()
        key = bucket(npix, P)
        shape = self.best.get(key)
        if shape is None:
            per = self.times.get(key, {})
            inflight = {}
            for k2, s, _, _ in self.pending:
                if k2 == key:
                    inflight[s] = inflight.get(s, 0) + 1
            shape = min(self.candidates, key=lambda s: len(per.get(s, ())) + inflight.get(s, 0))
        return shape, self.rasterizer(shape), key

    def start(self, stream=None):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def stop(self, key, shape: Shape, e0, stream=None):
        if key is None:
            return
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record(stream)
        self.pending.append((key, shape, e0, e1))

    def summary(self) -> dict:
        self._drain()
        return {f"{k[0]}:{k[1]}": s.label() for k, s in sorted(self.best.items())}
