"""One imaging problem on the device, with no host read-back in its step.

The step is the whole hot path of the method for one set of visibilities: Hankel kernel
generation for every |w|-plane (Section 4.3, Alg. 2; supports by the 1 % truncation rule of
Section 3.1, picked on the device), the oversampled cache laid out for the maximum support so
that the supports never have to come back to the host, gridding (Alg. 1 / Alg. 2) with the
launch shape the autotuner picked for this problem, and the dirty image (Section 3)
normalised by the weight sum the gridder accumulated, read on the device.  Plane values are
the means of equal-count chunks of the sorted |w| (Alg. 2 steps 1-3), computed once on the
device at set-up.

Everything here is argument marshalling around the C ABI (``api``); the benchmark's imaging
workload and its oracle parity test both run this class, so the tested step is the timed one.
"""
from __future__ import annotations

import torch

from . import api
from .api import Plan, WKernels
from .autotune import GRID_CHOICES, TILE_CHOICES, Autotuner


class Imager:
    def __init__(self, plan: Plan, taper: torch.Tensor, uvw: torch.Tensor, P: int, V_max: int | None = None,
                 w_planes: torch.Tensor | None = None):
        """plan: geometry and routes (trunc_frac > 0: supports by truncation on the device);
        taper: [R] float32; uvw: [3V] float32 (plane values come from its |w| unless given);
        P: number of |w|-planes; V_max: largest visibility count a step will grid."""
        dev = taper.device
        self.plan = plan
        self.taper = taper
        self.P = P
        self.w_planes = api.plane_values(uvw, P) if w_planes is None else w_planes
        V = int(uvw.numel() // 3) if V_max is None else int(V_max)
        self.V_max = V
        g = plan.geometry()
        self.ws = api.workspace(api.kernelgen_workspace_bytes(plan, P), dev)
        api.kernelgen_prepare(plan, P, self.ws)
        self.offsets = torch.tensor(api.kernel_layout_max(plan, P), dtype=torch.int64, device=dev)
        self.cache = torch.empty(int(self.offsets[-1].item()), dtype=torch.complex64, device=dev)
        self.support = torch.full((P,), plan.max_support, dtype=torch.int32, device=dev)
        self.radial = torch.empty((P, g.k_out), dtype=torch.complex64, device=dev)
        self.spline_m = torch.empty_like(self.radial) if plan.interp == "cubic" else None
        self.grid_ws = api.workspace(max(api.grid_workspace_bytes(plan.replace(grid_tile=t, grid_method=m), P, V)
                                         for m, t in list(GRID_CHOICES) + [(plan.grid_method, plan.grid_tile)]),
                                     dev)
        N = plan.image_size
        self.grid = torch.zeros((N, N), dtype=torch.complex64, device=dev)
        self.image = torch.empty((N, N), dtype=torch.float32, device=dev)
        self.stats = torch.zeros(2, dtype=torch.float64, device=dev)
        self.wk = WKernels(self.w_planes, self.support, self.offsets, self.cache, self.radial, self.spline_m)
        self.tuned = None

    # ------------------------------------------------------------------------- stages
    def kernels(self) -> None:
        """Radial lines, supports (truncation on the device) and the oversampled cache."""
        sup = self.support if self.plan.trunc_frac > 0 else None
        api.hankel_radial(self.plan, self.taper, self.w_planes, self.ws, self.radial, self.spline_m, sup)
        api.resample(self.plan, self.radial, self.spline_m, self.support, self.offsets, self.cache)

    def grid_only(self, uvw: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor | None = None) -> None:
        self.grid.zero_()
        self.stats.zero_()
        api.grid(self.plan, self.wk, uvw, vis, weight, self.grid, self.grid_ws, self.stats)

    def image_only(self) -> torch.Tensor:
        """Dirty image of the current grid (consumed), normalised by stats[0] on the device."""
        return api.dirty_image(self.plan, self.taper, self.grid, self.stats, self.image)

    def step(self, uvw: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor | None = None) -> torch.Tensor:
        """Kernel generation + gridding + dirty image, queued on the current stream."""
        self.kernels()
        self.grid_only(uvw, vis, weight)
        return self.image_only()

    # ----------------------------------------------------------------------- tuning
    def autotune(self, uvw: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor | None = None,
                 tuner: Autotuner | None = None, choices=None):
        """Pick the gridder's (method, tile) for this problem by timing every candidate on it;
        the kernels are generated first so that every candidate grids real taps."""
        tuner = tuner or Autotuner()
        self.kernels()
        N, P, V = self.plan.image_size, self.P, int(vis.numel())
        cands = [list(c) for c in (choices or GRID_CHOICES)]

        def run(c):
            self.grid.zero_()
            api.grid(self.plan.replace(grid_method=int(c[0]), grid_tile=int(c[1])), self.wk, uvw, vis, weight,
                     self.grid, self.grid_ws, self.stats)

        best = tuner.choose(Autotuner.key("grid", N, P, self.plan.max_support, V), cands, run)
        self.plan = self.plan.replace(grid_method=int(best[0]), grid_tile=int(best[1]))
        self.tuned = tuner
        return best


__all__ = ["Imager", "TILE_CHOICES"]
