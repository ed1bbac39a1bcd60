"""Python binding of the C ABI over torch CUDA tensors.

Functions carry the C names without the ``wp_`` prefix.  They check dtypes, devices and
contiguity, pass raw device pointers and the current torch stream to libwproj.so, and
allocate outputs with torch.  No numerical work happens here.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _lib

_ALIGN = 256


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, name: str, numel: int | None = None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t


@dataclasses.dataclass(frozen=True)
class Plan:
    """Imager settings (Section 5 of the paper); mirrors ``wp_plan``."""

    image_size: int
    cell_size: float
    oversampling: int = 8
    max_support: int = 15
    min_support: int = 3
    trunc_frac: float = 0.01
    radial_samples: int = 512
    interp: str = "cubic"
    kernelgen: str = "fp32"
    grid_tile: int = 0          # gridding tile side (0 = default 64; 32 or 64): tuning only
    grid_method: int = 3        # 3 row-owned shared tile (fastest measured), 0 register tile, 1/2/4: tuning only

    def c(self) -> _lib.WpPlan:
        return _lib.WpPlan(self.image_size, self.cell_size, self.oversampling, self.max_support,
                           self.min_support, self.trunc_frac, self.radial_samples,
                           _lib.INTERP[self.interp], _lib.KERNELGEN[self.kernelgen], self.grid_tile,
                           self.grid_method)

    def geometry(self) -> _lib.WpGeometry:
        g = _lib.WpGeometry()
        _lib.check("wp_plan_geometry", _lib.load().wp_plan_geometry(ctypes.byref(self.c()), ctypes.byref(g)))
        return g

    def replace(self, **kw) -> "Plan":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class WKernels:
    """A generated kernel set on the device (see ``wp_wkernels``)."""

    w_planes: torch.Tensor      # [P] float64
    support: torch.Tensor       # [P] int32
    offsets: torch.Tensor       # [P+1] int64
    cache: torch.Tensor         # [n] complex64
    radial: torch.Tensor | None = None     # [P][K_out] complex64
    spline_m: torch.Tensor | None = None   # [P][K_out] complex64

    @property
    def P(self) -> int:
        return int(self.w_planes.numel())

    def c(self) -> _lib.WpWkernels:
        return _lib.WpWkernels(self.P, 0, self.w_planes.data_ptr(), self.support.data_ptr(),
                               self.offsets.data_ptr(),
                               self.cache.data_ptr() if self.cache is not None else None,
                               self.radial.data_ptr() if self.radial is not None else None,
                               self.spline_m.data_ptr() if self.spline_m is not None else None)

    def subkernel(self, p: int, os_: int, support_host=None) -> torch.Tensor:
        s = int(self.support[p]) if support_host is None else int(support_host[p])
        a, b = int(self.offsets[p]), int(self.offsets[p + 1])
        W = 2 * s + 1
        return self.cache[a:a + os_ * os_ * W * W].view(os_, os_, W, W)


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A byte tensor usable as library scratch (torch allocations are 512-byte aligned)."""
    t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")
    if t.data_ptr() % _ALIGN:
        raise RuntimeError("workspace allocation is not 256-byte aligned")
    return t


# ------------------------------------------------------------------------------- layout
def kernel_layout(plan: Plan, support) -> list[int]:
    sup = (ctypes.c_int32 * len(support))(*[int(s) for s in support])
    off = (ctypes.c_int64 * (len(support) + 1))()
    _lib.check("wp_kernel_layout", _lib.load().wp_kernel_layout(ctypes.byref(plan.c()), len(support), sup, off))
    return list(off)


def kernel_layout_max(plan: Plan, P: int) -> list[int]:
    off = (ctypes.c_int64 * (P + 1))()
    _lib.check("wp_kernel_layout_max", _lib.load().wp_kernel_layout_max(ctypes.byref(plan.c()), P, off))
    return list(off)


# --------------------------------------------------------------------- kernel generation
def kernelgen_workspace_bytes(plan: Plan, P: int) -> int:
    return int(_lib.load().wp_kernelgen_workspace_bytes(ctypes.byref(plan.c()), P))


def kernelgen_prepare(plan: Plan, P: int, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    nbytes = kernelgen_workspace_bytes(plan, P)
    if ws is None:
        ws = workspace(nbytes)
    _need(ws, torch.uint8, "workspace")
    _lib.check("wp_kernelgen_prepare", _lib.load().wp_kernelgen_prepare(
        ctypes.byref(plan.c()), P, _ptr(ws), ws.numel(), _stream(stream)))
    return ws


def hankel_radial(plan: Plan, taper: torch.Tensor, w_planes: torch.Tensor, ws: torch.Tensor,
                  radial: torch.Tensor | None = None, spline_m: torch.Tensor | None = None,
                  support: torch.Tensor | None = None, stream=None):
    """Radial kernel lines (+ spline second derivatives, + supports when truncating)."""
    g = plan.geometry()
    P = int(w_planes.numel())
    _need(taper, torch.float32, "taper", plan.radial_samples)
    _need(w_planes, torch.float64, "w_planes")
    dev = taper.device
    if radial is None:
        radial = torch.empty((P, g.k_out), dtype=torch.complex64, device=dev)
    if spline_m is None and plan.interp == "cubic":
        spline_m = torch.empty((P, g.k_out), dtype=torch.complex64, device=dev)
    if support is None and plan.trunc_frac > 0:
        support = torch.empty(P, dtype=torch.int32, device=dev)
    _lib.check("wp_hankel_radial", _lib.load().wp_hankel_radial(
        ctypes.byref(plan.c()), _ptr(taper), _ptr(w_planes), P, _ptr(ws), ws.numel(), _ptr(radial),
        _ptr(spline_m), _ptr(support), _stream(stream)))
    return radial, spline_m, support


def resample(plan: Plan, radial: torch.Tensor, spline_m: torch.Tensor | None, support: torch.Tensor,
             offsets: torch.Tensor, cache: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    P = int(support.numel())
    _need(radial, torch.complex64, "radial")
    _need(support, torch.int32, "support")
    _need(offsets, torch.int64, "offsets", P + 1)
    if cache is None:
        cache = torch.empty(int(offsets[-1].item()), dtype=torch.complex64, device=radial.device)
    _lib.check("wp_resample", _lib.load().wp_resample(
        ctypes.byref(plan.c()), _ptr(radial), _ptr(spline_m), P, _ptr(support), _ptr(offsets),
        _ptr(cache), _stream(stream)))
    return cache


def make_wkernels(plan: Plan, taper: torch.Tensor, w_planes, supports=None,
                  ws: torch.Tensor | None = None, prepare: bool = True, stream=None) -> WKernels:
    """Hankel w-kernels of every plane (Alg. 2).  With ``supports`` given (or
    ``plan.trunc_frac <= 0``) the layout is compact and nothing is read back; otherwise the
    1 % truncation supports are read back to lay the cache out compactly."""
    dev = taper.device
    w_planes = torch.as_tensor(w_planes, dtype=torch.float64, device=dev).contiguous()
    wp_host = w_planes.cpu()
    if (wp_host < 0).any() or (wp_host[1:] < wp_host[:-1]).any():
        raise ValueError("w_planes must be ascending and >= 0 (|w| planes)")
    P = int(w_planes.numel())
    if ws is None:
        ws = workspace(kernelgen_workspace_bytes(plan, P), dev)
        prepare = True
    if prepare:
        kernelgen_prepare(plan, P, ws, stream)
    if supports is not None:
        sup_host = [int(s) for s in supports]
        off = torch.tensor(kernel_layout(plan, sup_host), dtype=torch.int64, device=dev)
        sup = torch.tensor(sup_host, dtype=torch.int32, device=dev)
        p_fixed = plan.replace(trunc_frac=0.0)
        radial, spline_m, _ = hankel_radial(p_fixed, taper, w_planes, ws, stream=stream)
        cache = resample(p_fixed, radial, spline_m, sup, off, stream=stream)
        return WKernels(w_planes, sup, off, cache, radial, spline_m)
    if plan.trunc_frac <= 0:
        raise ValueError("supports are required when plan.trunc_frac <= 0")
    radial, spline_m, sup = hankel_radial(plan, taper, w_planes, ws, stream=stream)
    sup_host = sup.cpu().tolist()
    off = torch.tensor(kernel_layout(plan, sup_host), dtype=torch.int64, device=dev)
    cache = resample(plan, radial, spline_m, sup, off, stream=stream)
    return WKernels(w_planes, sup, off, cache, radial, spline_m)


class OwnedWKernels:
    """A kernel set in device memory the library allocated (``wp_make_wkernels_owned``):
    usable wherever a ``WKernels`` is (gridding, degridding); released by ``free()`` or when
    the object is collected."""

    def __init__(self, kc: _lib.WpWkernels):
        self._kc = kc

    @property
    def P(self) -> int:
        return int(self._kc.P)

    def c(self) -> _lib.WpWkernels:
        if not self._kc.flags:
            raise RuntimeError("kernel set already freed")
        return self._kc

    def free(self) -> None:
        if self._kc.flags:
            _lib.check("wp_free_kernels", _lib.load().wp_free_kernels(ctypes.byref(self._kc)))

    def __del__(self):
        try:
            self.free()
        except Exception:   # interpreter or CUDA teardown: the process releases the memory
            pass


def make_wkernels_owned(plan: Plan, taper: torch.Tensor, w_planes, supports=None, stream=None) -> OwnedWKernels:
    """The kernels of ``make_wkernels`` in library-allocated device memory, from host plane
    values (ascending, >= 0) and, with ``plan.trunc_frac <= 0``, host supports."""
    _need(taper, torch.float32, "taper", plan.radial_samples)
    w = torch.as_tensor(w_planes, dtype=torch.float64).contiguous().cpu()
    sup = None if supports is None else torch.as_tensor(supports, dtype=torch.int32).contiguous().cpu()
    kc = _lib.WpWkernels()
    _lib.check("wp_make_wkernels_owned", _lib.load().wp_make_wkernels_owned(
        ctypes.byref(plan.c()), _ptr(taper), ctypes.c_void_p(w.data_ptr()), int(w.numel()),
        None if sup is None else ctypes.c_void_p(sup.data_ptr()), ctypes.byref(kc), _stream(stream)))
    return OwnedWKernels(kc)


def fft_wkernels(plan: Plan, taper: torch.Tensor, w_planes, supports, circular: bool = True,
                 ws: torch.Tensor | None = None, stream=None) -> WKernels:
    """Kernel cache by the standard 2D-FFT route (Alg. 1 with workspace undersampling),
    for comparison with the Hankel route; supports are given."""
    dev = taper.device
    _need(taper, torch.float32, "taper", plan.radial_samples)
    w_planes = torch.as_tensor(w_planes, dtype=torch.float64, device=dev).contiguous()
    P = int(w_planes.numel())
    sup_host = [int(s) for s in supports]
    off = torch.tensor(kernel_layout(plan, sup_host), dtype=torch.int64, device=dev)
    sup = torch.tensor(sup_host, dtype=torch.int32, device=dev)
    if ws is None:
        ws = workspace(int(_lib.load().wp_fft_workspace_bytes(ctypes.byref(plan.c()), P)), dev)
    cache = torch.empty(int(off[-1].item()), dtype=torch.complex64, device=dev)
    _lib.check("wp_fft_wkernels", _lib.load().wp_fft_wkernels(
        ctypes.byref(plan.c()), _ptr(taper), _ptr(w_planes), P, _ptr(sup), _ptr(off), int(bool(circular)),
        _ptr(ws), ws.numel(), _ptr(cache), _stream(stream)))
    return WKernels(w_planes, sup, off, cache)


def plane_values(uvw: torch.Tensor, P: int, stream=None) -> torch.Tensor:
    """|w|-plane values: means of P equal-count chunks of the sorted |w| (Alg. 2 steps 1-3)."""
    V = int(uvw.numel() // 3)
    _need(uvw, torch.float32, "uvw", 3 * V)
    ws = workspace(int(_lib.load().wp_plane_values_workspace_bytes(V)), uvw.device)
    out = torch.empty(P, dtype=torch.float64, device=uvw.device)
    _lib.check("wp_plane_values", _lib.load().wp_plane_values(
        _ptr(uvw), V, P, _ptr(ws), ws.numel(), _ptr(out), _stream(stream)))
    return out


# ----------------------------------------------------------------------------- gridding
def grid_workspace_bytes(plan: Plan, P: int, V: int) -> int:
    return int(_lib.load().wp_grid_workspace_bytes(ctypes.byref(plan.c()), P, V))


def grid(plan: Plan, wk: WKernels, uvw: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor | None = None,
         out: torch.Tensor | None = None, ws: torch.Tensor | None = None, stats: torch.Tensor | None = None,
         stream=None):
    """Grid visibilities (accumulating into ``out``); returns (grid, stats) with
    stats = [sum of gridded weights, number dropped] (float64, device)."""
    V = int(vis.numel())
    _need(uvw, torch.float32, "uvw", 3 * V)
    _need(vis, torch.complex64, "vis")
    if weight is not None:
        _need(weight, torch.float32, "weight", V)
    N = plan.image_size
    dev = vis.device
    if out is None:
        out = torch.zeros((N, N), dtype=torch.complex64, device=dev)
    _need(out, torch.complex64, "grid", N * N)
    if ws is None:
        ws = workspace(grid_workspace_bytes(plan, wk.P, V), dev)
    if stats is None:
        stats = torch.zeros(2, dtype=torch.float64, device=dev)
    kc = wk.c()
    _lib.check("wp_grid", _lib.load().wp_grid(
        ctypes.byref(plan.c()), ctypes.byref(kc), _ptr(uvw), _ptr(vis), _ptr(weight), V, _ptr(ws),
        ws.numel(), _ptr(out), _ptr(stats), _stream(stream)))
    return out, stats


def degrid(plan: Plan, wk: WKernels, uvw: torch.Tensor, grid_: torch.Tensor, out: torch.Tensor | None = None,
           ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    V = int(uvw.numel() // 3)
    _need(uvw, torch.float32, "uvw", 3 * V)
    N = plan.image_size
    _need(grid_, torch.complex64, "grid", N * N)
    dev = uvw.device
    if out is None:
        out = torch.empty(V, dtype=torch.complex64, device=dev)
    if ws is None:
        ws = workspace(grid_workspace_bytes(plan, wk.P, V), dev)
    kc = wk.c()
    _lib.check("wp_degrid", _lib.load().wp_degrid(
        ctypes.byref(plan.c()), ctypes.byref(kc), _ptr(uvw), _ptr(grid_), V, _ptr(ws), ws.numel(),
        _ptr(out), _stream(stream)))
    return out


def dirty_image(plan: Plan, taper: torch.Tensor, grid_: torch.Tensor, weight_sum,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Dirty image; ``grid_`` is transformed in place (consumed).  ``weight_sum`` is a host
    number, or a float64 CUDA tensor whose first element is read on the device -- normally the
    ``stats`` that ``grid`` returned (``stats[0]`` = sum of the weights actually gridded), which
    keeps the normalisation free of host read-backs."""
    N = plan.image_size
    _need(taper, torch.float32, "taper", plan.radial_samples)
    _need(grid_, torch.complex64, "grid", N * N)
    if out is None:
        out = torch.empty((N, N), dtype=torch.float32, device=grid_.device)
    if isinstance(weight_sum, torch.Tensor):
        _need(weight_sum, torch.float64, "weight_sum")
        _lib.check("wp_dirty_image_stats", _lib.load().wp_dirty_image_stats(
            ctypes.byref(plan.c()), _ptr(taper), _ptr(grid_), _ptr(weight_sum), _ptr(out), _stream(stream)))
        return out
    _lib.check("wp_dirty_image", _lib.load().wp_dirty_image(
        ctypes.byref(plan.c()), _ptr(taper), _ptr(grid_), float(weight_sum), _ptr(out), _stream(stream)))
    return out


def image_to_grid(plan: Plan, taper: torch.Tensor, image: torch.Tensor, weight_sum: float,
                  out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    N = plan.image_size
    _need(taper, torch.float32, "taper", plan.radial_samples)
    _need(image, torch.float32, "image", N * N)
    if out is None:
        out = torch.empty((N, N), dtype=torch.complex64, device=image.device)
    _lib.check("wp_image_to_grid", _lib.load().wp_image_to_grid(
        ctypes.byref(plan.c()), _ptr(taper), _ptr(image), float(weight_sum), _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------------ persistent batches
@dataclasses.dataclass
class GridJob:
    """One job of ``grid_batch``: the arguments of one ``grid`` call (workspace and stats
    tensors included; the workspace must be sized for grid_method 3)."""

    plan: Plan
    wk: "WKernels | OwnedWKernels"
    uvw: torch.Tensor
    vis: torch.Tensor
    weight: torch.Tensor | None
    grid: torch.Tensor
    ws: torch.Tensor
    stats: torch.Tensor | None = None


def grid_batch_workspace(device=None) -> torch.Tensor:
    return workspace(int(_lib.load().wp_grid_batch_workspace_bytes()), device)


def _job_array(jobs: list[GridJob]):
    arr = (_lib.WpGridJob * len(jobs))()
    for i, j in enumerate(jobs):
        V = int(j.vis.numel())
        _need(j.uvw, torch.float32, "uvw", 3 * V)
        _need(j.vis, torch.complex64, "vis")
        if j.weight is not None:
            _need(j.weight, torch.float32, "weight", V)
        _need(j.grid, torch.complex64, "grid", j.plan.image_size ** 2)
        _need(j.ws, torch.uint8, "workspace")
        arr[i] = _lib.WpGridJob(j.plan.c(), j.wk.c(), j.uvw.data_ptr(), j.vis.data_ptr(),
                                j.weight.data_ptr() if j.weight is not None else None, V, j.ws.data_ptr(),
                                j.ws.numel(), j.grid.data_ptr(),
                                j.stats.data_ptr() if j.stats is not None else None)
    return arr


def grid_batch(jobs: list[GridJob], bws: torch.Tensor, stream=None, fused: bool = False) -> None:
    """Grid every job in persistent launches pulling work from one device queue per gridder kind
    (see ``wp_grid_batch``; ``fused``: ``wp_grid_batch_fused``, orderings and items in one
    launch with bounded waits); each job's grid and stats as ``grid`` would leave them.  Order
    the jobs largest first."""
    arr = _job_array(jobs)
    name = "wp_grid_batch_fused" if fused else "wp_grid_batch"
    _lib.check(name, getattr(_lib.load(), name)(len(jobs), arr, _ptr(bws), bws.numel(), _stream(stream)))


def grid_batch_status(bws: torch.Tensor, stream=None) -> int:
    st = ctypes.c_int32()
    _lib.check("wp_grid_batch_status", _lib.load().wp_grid_batch_status(_ptr(bws), ctypes.byref(st),
                                                                        _stream(stream)))
    return int(st.value)


def grid_batch_selftest(jobs: list[GridJob], bws: torch.Tensor, stream=None) -> int:
    """Runs the batch with its scatter withheld so that every gridding wait expires; returns
    the device status (WP_ERR_TIMEOUT = -6 expected)."""
    arr = _job_array(jobs)
    st = ctypes.c_int32()
    _lib.check("wp_grid_batch_selftest", _lib.load().wp_grid_batch_selftest(
        len(jobs), arr, _ptr(bws), bws.numel(), ctypes.byref(st), _stream(stream)))
    return int(st.value)
