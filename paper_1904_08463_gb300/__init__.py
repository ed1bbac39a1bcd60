"""GB300 (sm_103a) implementation of Hankel-accelerated w-projection.

Lucas, Skipper & Scaife, "Fast W-Projection for Wide-field Imaging" (MNRAS 2019):
w-kernels by an order-0 Hankel transform (Section 4.3, Alg. 2), convolutional gridding,
degridding and dirty imaging.  All computation runs in libwproj.so (hand-written CUDA
behind the C ABI of include/wproj.h); this package only marshals torch tensors.
"""
from .api import (OwnedWKernels, Plan, WKernels, degrid, dirty_image, fft_wkernels, grid, grid_workspace_bytes,
                  hankel_radial, image_to_grid, kernel_layout, plane_values, kernel_layout_max, kernelgen_prepare,
                  kernelgen_workspace_bytes, make_wkernels, make_wkernels_owned, resample, workspace)
from ._lib import WPError

__all__ = ["OwnedWKernels", "Plan", "WKernels", "WPError", "degrid", "dirty_image", "fft_wkernels", "grid", "grid_workspace_bytes",
           "hankel_radial", "image_to_grid", "kernel_layout", "kernel_layout_max", "kernelgen_prepare",
           "kernelgen_workspace_bytes", "make_wkernels", "make_wkernels_owned", "plane_values", "resample", "workspace"]
