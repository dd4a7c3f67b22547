"""GB300-native w-projection convolutional gridding and degridding with compression.

The method is the WImager algorithm of D. Muscat, "High-Performance Image Synthesis for
Radio Interferometry" (arXiv:1403.4209): convolutional gridding with w-projection kernels
(Sec. 2.1-2.2), the thesis's compression of consecutive records (Sec. 4.3.3), its kernel
generator (Sec. 4.2) and image finaliser (Sec. 4.7), plus degridding as the exact adjoint.

All computation runs in the CUDA library libwgrid.so (include/wgrid.h); this package only
marshals torch tensors into its C ABI.
"""
from ._lib import CONST, WgError, header_functions, lib
from .api import (DEGRID_ADJOINT, DEGRID_PREDICT, IMAGE_PER_POL, IMAGE_PER_POL_RAW, IMAGE_STOKES_CIRCULAR, IMAGE_STOKES_I,
                  IMAGE_STOKES_LINEAR, IMAGE_TRANSPOSE, IMAGE_WSTACK,
                  ConvTable, Grid, VisBatch, WorkList, ceiling, degrid_vis, grid_autotune, grid_correct, grid_vis, vis_weight, image_to_grid, launch_count,
                  vis_compress)
from .autograd import DegridFn, SkyModel

__all__ = [
    "CONST", "WgError", "header_functions", "lib", "DEGRID_ADJOINT", "DEGRID_PREDICT", "IMAGE_PER_POL",
    "IMAGE_STOKES_I", "IMAGE_PER_POL_RAW", "IMAGE_TRANSPOSE", "IMAGE_STOKES_LINEAR", "IMAGE_STOKES_CIRCULAR", "IMAGE_WSTACK", "ConvTable", "Grid", "VisBatch", "WorkList",
    "ceiling", "degrid_vis", "grid_autotune", "grid_correct", "vis_weight", "grid_vis", "image_to_grid", "launch_count", "vis_compress", "DegridFn", "SkyModel",
]
