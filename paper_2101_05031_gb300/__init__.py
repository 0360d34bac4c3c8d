"""GB300-native slicer for convolution-surface lattices (arxiv 2101.05031).

The compute path is libcslice.so (hand-written CUDA for sm_103a, C ABI in
include/cslice.h). This package only marshals arguments to it.
"""
from ._lib import CslError, load  # noqa: F401
from .batch import Batch  # noqa: F401
from .density import density_match, support_optimize  # noqa: F401
from .slicer import ContourSet, DeviceContours, Lattice, last_stats, measure_fp32_peak  # noqa: F401

__all__ = ["Lattice", "Batch", "density_match", "support_optimize", "ContourSet", "DeviceContours", "CslError", "load", "last_stats",
           "volume_fraction", "volume_fraction_backward", "VolumeFraction"]


def __getattr__(name):
    # the volume-fraction layer needs torch; import it on first use
    if name in ("volume_fraction", "volume_fraction_backward", "VolumeFraction", "cells_desc"):
        from . import vf
        return getattr(vf, name)
    raise AttributeError(name)
