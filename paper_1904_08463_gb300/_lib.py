"""ctypes view of libwproj.so (the C ABI declared in include/wproj.h).

Argument marshalling only: every computation happens in the CUDA library.  Loading fails
loudly when the library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwproj.so")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_double = ctypes.c_double
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p

WP_OK = 0
ERRORS = {
    -1: "WP_ERR_NULL", -2: "WP_ERR_SIZE", -3: "WP_ERR_PLAN", -4: "WP_ERR_WORKSPACE",
    -5: "WP_ERR_CUDA", -6: "WP_ERR_TIMEOUT", -7: "WP_ERR_DEVICE", -8: "WP_ERR_UNSUPPORTED",
}
INTERP = {"cubic": 0, "linear": 1}
KERNELGEN = {"fp32": 0, "tf32x3": 1, "projslice": 2, "bf16x3": 3, "bf16x6": 4}


class WpPlan(ctypes.Structure):
    _fields_ = [
        ("image_size", c_int32),
        ("cell_size", c_double),
        ("oversampling", c_int32),
        ("max_support", c_int32),
        ("min_support", c_int32),
        ("trunc_frac", c_double),
        ("radial_samples", c_int32),
        ("interp", c_int32),
        ("kernelgen", c_int32),
        ("grid_tile", c_int32),
        ("grid_method", c_int32),
    ]


class WpGeometry(ctypes.Structure):
    _fields_ = [
        ("k_out", c_int32),
        ("r_pad", c_int32),
        ("fft_workspace", c_int32),
        ("reserved", c_int32),
        ("du", c_double),
        ("r_max", c_double),
    ]


class WpWkernels(ctypes.Structure):
    _fields_ = [
        ("P", c_int32),
        ("flags", c_int32),
        ("w_planes", c_void_p),
        ("support", c_void_p),
        ("offsets", c_void_p),
        ("cache", c_void_p),
        ("radial", c_void_p),
        ("spline_m", c_void_p),
    ]


class WpGridJob(ctypes.Structure):
    _fields_ = [
        ("plan", WpPlan),
        ("kernels", WpWkernels),
        ("uvw", c_void_p),
        ("vis", c_void_p),
        ("weight", c_void_p),
        ("V", c_int64),
        ("workspace", c_void_p),
        ("workspace_bytes", c_size_t),
        ("grid", c_void_p),
        ("stats", c_void_p),
    ]


GRID_BATCH_MAX_JOBS = 128


class WPError(RuntimeError):
    def __init__(self, fn: str, code: int, detail: str = ""):
        self.code = code
        msg = f"{fn} failed: {ERRORS.get(code, code)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


P_ = ctypes.POINTER
_SIGS = {
    "wp_version": (c_int32, []),
    "wp_strerror": (ctypes.c_char_p, [c_int32]),
    "wp_make_wkernels_owned": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_int32, c_void_p, P_(WpWkernels),
                                         c_void_p]),
    "wp_free_kernels": (c_int32, [P_(WpWkernels)]),
    "wp_last_error_string": (ctypes.c_char_p, []),
    "wp_release": (None, []),
    "wp_plan_geometry": (c_int32, [P_(WpPlan), P_(WpGeometry)]),
    "wp_kernel_layout": (c_int32, [P_(WpPlan), c_int32, c_void_p, c_void_p]),
    "wp_kernel_layout_max": (c_int32, [P_(WpPlan), c_int32, c_void_p]),
    "wp_kernelgen_workspace_bytes": (c_size_t, [P_(WpPlan), c_int32]),
    "wp_kernelgen_prepare": (c_int32, [P_(WpPlan), c_int32, c_void_p, c_size_t, c_void_p]),
    "wp_hankel_radial": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_int32, c_void_p, c_size_t,
                                   c_void_p, c_void_p, c_void_p, c_void_p]),
    "wp_kernelgen_status": (c_int32, [P_(WpPlan), c_int32, c_void_p, c_size_t, c_void_p, c_void_p]),
    "wp_selftest_bounded_wait": (c_int32, [P_(WpPlan), c_int32, c_void_p, c_size_t, c_void_p, c_void_p,
                                           c_void_p]),
    "wp_resample": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                              c_void_p, c_void_p]),
    "wp_make_wkernels": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                                   c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_void_p]),
    "wp_fft_workspace_bytes": (c_size_t, [P_(WpPlan), c_int32]),
    "wp_fft_wkernels": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                  c_void_p, c_size_t, c_void_p, c_void_p]),
    "wp_plane_values_workspace_bytes": (c_size_t, [c_int64]),
    "wp_plane_values": (c_int32, [c_void_p, c_int64, c_int32, c_void_p, c_size_t, c_void_p, c_void_p]),
    "wp_grid_workspace_bytes": (c_size_t, [P_(WpPlan), c_int32, c_int64]),
    "wp_grid": (c_int32, [P_(WpPlan), P_(WpWkernels), c_void_p, c_void_p, c_void_p, c_int64,
                          c_void_p, c_size_t, c_void_p, c_void_p, c_void_p]),
    "wp_grid_static": (c_int32, [P_(WpPlan), P_(WpWkernels), c_void_p, c_void_p, c_void_p, c_int64,
                                 c_void_p, c_void_p, c_void_p]),
    "wp_degrid": (c_int32, [P_(WpPlan), P_(WpWkernels), c_void_p, c_void_p, c_int64, c_void_p,
                            c_size_t, c_void_p, c_void_p]),
    "wp_grad_workspace_bytes": (c_size_t, [P_(WpPlan), c_int32, c_int64]),
    "wp_grad_radial": (c_int32, [P_(WpPlan), P_(WpWkernels), c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                 c_size_t, c_void_p, c_void_p, c_void_p]),
    "wp_hankel_adjoint": (c_int32, [P_(WpPlan), c_void_p, c_int32, c_void_p, c_size_t, c_void_p, c_void_p,
                                    c_void_p, c_void_p]),
    "wp_image_adjoint": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_void_p,
                                   c_void_p]),
    "wp_dirty_image": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_double, c_void_p, c_void_p]),
    "wp_dirty_image_stats": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "wp_grid_batch_workspace_bytes": (c_size_t, []),
    "wp_grid_batch": (c_int32, [c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "wp_grid_batch_fused": (c_int32, [c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "wp_grid_batch_status": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "wp_grid_batch_selftest": (c_int32, [c_int32, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "wp_probe_fp32_fma": (c_int32, [c_int32, c_int32, c_void_p, P_(c_double), c_void_p]),
    "wp_bounds_status": (c_int32, [P_(ctypes.c_uint64), c_int32]),
    "wp_probe_l2_taps": (c_int32, [c_void_p, c_int64, c_int32, c_int32, c_int32, c_void_p, P_(c_double), c_void_p]),
    "wp_image_to_grid": (c_int32, [P_(WpPlan), c_void_p, c_void_p, c_double, c_void_p, c_void_p]),
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libwproj.so.  Raises if it is missing: build it with
    ``python -c "import __graft_entry__ as g; g.build()"``."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: the CUDA library has not been built "
                                  "(run paper_1904_08463_gb300.build.build())")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(fn_name: str, code: int) -> None:
    if code != WP_OK:
        detail = ""
        try:
            detail = (load().wp_last_error_string() or b"").decode()
        except Exception:
            pass
        raise WPError(fn_name, code, detail)
