"""GB300-native differentiable 3D Gaussian Splatting rasterizer (forward, backward, SE(3) pose
gradient, batched multi-view / multi-scene launches, fused losses and in-kernel Adam).

The compute lives in libgs (include/gs.h, built from csrc/ for sm_103a); this package is its thin
Python binding.  Importing the binding loads libgs and raises if it is unavailable.
"""
from . import scenes  # noqa: F401  (input generators; no rasterizer arithmetic)

__all__ = ["scenes", "raster", "load"]


def load():
    """Load libgs and return the torch-facing binding module."""
    from . import raster
    raster.L.load()
    return raster
