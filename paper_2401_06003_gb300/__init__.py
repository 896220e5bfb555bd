"""GB300-native differentiable trilinear point splatting (the TRIPS render path).

The compute lives in ``libtrips.so`` (CUDA for sm_103a, C ABI in
``include/trips.h``); this package builds it in-tree, binds it with ctypes
and exposes a ``torch.autograd.Function`` over it.
"""
from . import scenes  # noqa: F401
from ._lib import TripsError, load  # noqa: F401
from .splat import (BatchRenderer, Frame, Renderer, TripsSplat, autotune_batch_tiles, autotune_tiles,  # noqa: F401
                    init_point_sizes, permute_rows, spatial_order, splat)

__all__ = ["Renderer", "BatchRenderer", "autotune_tiles", "autotune_batch_tiles", "init_point_sizes", "spatial_order", "permute_rows", "TripsSplat", "splat", "Frame", "TripsError", "load", "scenes"]
