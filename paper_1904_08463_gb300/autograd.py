"""Differentiable visibility prediction: torch.autograd.Function over the C ABI.

    V = degrid(K(t), image_to_grid(I; t))

for a real model image I [N][N] and the radial anti-aliasing taper t [R] (the kernels K(t)
are the Hankel w-kernels of Section 4.3 for fixed plane values and supports).  The
backward pass is hand-written in CUDA: the image gradient is the dirty image of the
gridded visibility gradient (gridding is the adjoint of degridding), and the taper gradient
goes through the adjoint of the resample/spline steps and the transposed Hankel matrix,
plus the taper's own appearance in the image-to-grid step.  A chi-squared data term
sum_k w_k |V_k - V_obs,k|^2 built on the output in torch gives both gradients.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .api import (Plan, WKernels, _need, _ptr, _stream, degrid, grid, grid_workspace_bytes,
                  hankel_radial, image_to_grid, kernel_layout, kernelgen_prepare,
                  kernelgen_workspace_bytes, resample, workspace)


class Predictor:
    """Fixed geometry of a differentiable prediction: plan, |w|-plane values, supports and
    visibility coordinates, with the device workspaces reused across calls."""

    def __init__(self, plan: Plan, w_planes, supports, uvw: torch.Tensor, weight_sum: float = 1.0,
                 degrid_method: int | None = None):
        """degrid_method: the degridder of the forward prediction (a ``grid_method``; default the
        plan's own); the backward pass grids with the plan's method."""
        if plan.trunc_frac > 0:
            plan = plan.replace(trunc_frac=0.0)
        self.plan = plan
        self.degrid_plan = plan if degrid_method is None else plan.replace(grid_method=int(degrid_method))
        dev = uvw.device
        self.uvw = _need(uvw.reshape(-1), torch.float32, "uvw")
        self.V = self.uvw.numel() // 3
        self.w_planes = torch.as_tensor(w_planes, dtype=torch.float64, device=dev).contiguous()
        self.P = int(self.w_planes.numel())
        sup = [int(s) for s in supports]
        self.support = torch.tensor(sup, dtype=torch.int32, device=dev)
        self.offsets = torch.tensor(kernel_layout(plan, sup), dtype=torch.int64, device=dev)
        self.kg_ws = workspace(kernelgen_workspace_bytes(plan, self.P), dev)
        kernelgen_prepare(plan, self.P, self.kg_ws)
        self.grid_ws = workspace(max(grid_workspace_bytes(plan, self.P, self.V),
                                     grid_workspace_bytes(self.degrid_plan, self.P, self.V),
                                     int(_lib.load().wp_grad_workspace_bytes(ctypes.byref(plan.c()), self.P,
                                                                             self.V))), dev)
        self.weight_sum = float(weight_sum)

    def kernels(self, taper: torch.Tensor) -> WKernels:
        radial, spline_m, _ = hankel_radial(self.plan, taper, self.w_planes, self.kg_ws)
        cache = resample(self.plan, radial, spline_m, self.support, self.offsets)
        return WKernels(self.w_planes, self.support, self.offsets, cache, radial, spline_m)

    def __call__(self, image: torch.Tensor, taper: torch.Tensor) -> torch.Tensor:
        return Visibilities.apply(image, taper, self)


class Visibilities(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image: torch.Tensor, taper: torch.Tensor, pr: Predictor):
        image = _need(image.detach().contiguous(), torch.float32, "image")
        taper = _need(taper.detach().contiguous(), torch.float32, "taper")
        wk = pr.kernels(taper)
        G = image_to_grid(pr.plan, taper, image, pr.weight_sum)
        vis = degrid(pr.degrid_plan, wk, pr.uvw, G, ws=pr.grid_ws)
        ctx.pr = pr
        ctx.wk = wk
        ctx.save_for_backward(image, taper, G)
        return vis

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        image, taper, G = ctx.saved_tensors
        pr: Predictor = ctx.pr
        wk: WKernels = ctx.wk
        g = g.contiguous().to(torch.complex64)
        lib = _lib.load()
        plan_c = pr.plan.c()
        dev = image.device
        grad_taper = torch.zeros_like(taper)
        grad_image = torch.empty_like(image)
        need_t = ctx.needs_input_grad[1]
        if need_t:
            gC = torch.empty_like(wk.radial)
            gM = torch.empty_like(wk.radial)
            kc = wk.c()
            _lib.check("wp_grad_radial", lib.wp_grad_radial(
                ctypes.byref(plan_c), ctypes.byref(kc), _ptr(pr.uvw), _ptr(g), _ptr(G), pr.V, _ptr(pr.grid_ws),
                pr.grid_ws.numel(), _ptr(gC), _ptr(gM), _stream()))
            _lib.check("wp_hankel_adjoint", lib.wp_hankel_adjoint(
                ctypes.byref(plan_c), _ptr(pr.w_planes), pr.P, _ptr(pr.kg_ws), pr.kg_ws.numel(), _ptr(gC),
                _ptr(gM), _ptr(grad_taper), _stream()))
        Gg, _ = grid(pr.plan, wk, pr.uvw, g, None, ws=pr.grid_ws)
        _lib.check("wp_image_adjoint", lib.wp_image_adjoint(
            ctypes.byref(plan_c), _ptr(taper), _ptr(image), _ptr(Gg), pr.weight_sum, _ptr(grad_image),
            _ptr(grad_taper), _stream()))
        return (grad_image if ctx.needs_input_grad[0] else None, grad_taper if need_t else None, None)


def chi2(vis_model: torch.Tensor, vis_obs: torch.Tensor, weight: torch.Tensor | None = None) -> torch.Tensor:
    """Data-fidelity term sum_k w_k |V_k - V_obs,k|^2 (float64 accumulation)."""
    r = (vis_model - vis_obs).to(torch.complex128)
    a = r.real ** 2 + r.imag ** 2
    if weight is not None:
        a = a * weight.to(torch.float64)
    return a.sum()
