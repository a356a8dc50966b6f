"""GB300-native differentiable tile rasterizer for DashGaussian's scheduled
3DGS optimisation (arXiv 2503.18402).

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/dashgs.h``); ``capi`` loads it and fails loudly when it is missing.
``synth`` draws seeded synthetic inputs and does not touch the library.
"""
__all__ = ["capi", "raster", "train", "synth"]
