"""The C ABI library loads, exports every function declared in include/wproj.h, and its
host-side logic (plan validation, layouts, argument checks) behaves as documented.
No device work is requested here."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_1904_08463_gb300 import _lib, build

    if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
        build.build()
    return _lib, _lib.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "wproj.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(wp_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol():
    _, lib = _lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_plan_geometry():
    L, lib = _lib()
    import numpy as np

    p = L.WpPlan(256, float(np.deg2rad(2.0) / 256), 8, 15, 3, 0.01, 512, 0, 0, 0, 0)
    g = L.WpGeometry()
    assert lib.wp_plan_geometry(ctypes.byref(p), ctypes.byref(g)) == 0
    assert g.k_out == 256 and g.r_pad == 512 and g.fft_workspace == 32
    assert g.du == pytest.approx(1.0 / np.deg2rad(2.0), rel=1e-15)
    assert g.r_max == pytest.approx(np.deg2rad(1.0), rel=1e-15)
    p2 = L.WpPlan(4096, float(np.deg2rad(8.0) / 4096), 8, 127, 7, 0.0, 4096, 0, 1, 32, 1)
    assert lib.wp_plan_geometry(ctypes.byref(p2), ctypes.byref(g)) == 0
    assert g.k_out == 1152 and g.fft_workspace == 256


def test_every_named_route_is_a_valid_plan():
    """Each kernel-generation route the binding names (FP32, TF32x3, projection slice, BF16x3,
    BF16x6) is accepted, and the workspace does not depend on the route."""
    L, lib = _lib()
    sizes = set()
    for name, code in L.KERNELGEN.items():
        p = L.WpPlan(256, 1e-4, 8, 15, 3, 0.01, 512, 0, code, 0, 0)
        g = L.WpGeometry()
        assert lib.wp_plan_geometry(ctypes.byref(p), ctypes.byref(g)) == 0, name
        sizes.add(lib.wp_kernelgen_workspace_bytes(ctypes.byref(p), 100))
    assert sorted(L.KERNELGEN.values()) == [0, 1, 2, 3, 4]
    assert len(sizes) == 1 and sizes.pop() > 0


@pytest.mark.parametrize("field,value", [("image_size", 255), ("image_size", 8), ("cell_size", 0.0),
                                         ("cell_size", 0.01), ("oversampling", 0), ("oversampling", 17),
                                         ("max_support", 0), ("max_support", 200), ("min_support", 16),
                                         ("radial_samples", 4), ("interp", 2), ("kernelgen", 5), ("kernelgen", -1),
                                         ("trunc_frac", 1.0), ("grid_tile", 48),
                                         ("grid_method", 10), ("grid_method", -1)])
def test_invalid_plans_rejected(field, value):
    L, lib = _lib()
    p = L.WpPlan(256, 1e-4, 8, 15, 3, 0.01, 512, 0, 0, 0, 0)
    setattr(p, field, value)
    g = L.WpGeometry()
    assert lib.wp_plan_geometry(ctypes.byref(p), ctypes.byref(g)) == -3


def test_layout_and_argument_errors():
    L, lib = _lib()
    p = L.WpPlan(256, 1e-4, 8, 15, 3, 0.01, 512, 0, 0, 0, 0)
    sup = (ctypes.c_int32 * 3)(3, 5, 15)
    off = (ctypes.c_int64 * 4)()
    assert lib.wp_kernel_layout(ctypes.byref(p), 3, sup, off) == 0
    assert list(off) == [0, 64 * 49, 64 * (49 + 121), 64 * (49 + 121 + 961)]
    bad = (ctypes.c_int32 * 1)(16)
    assert lib.wp_kernel_layout(ctypes.byref(p), 1, bad, off) == -2
    assert lib.wp_kernel_layout_max(ctypes.byref(p), 2, off) == 0
    assert list(off)[:3] == [0, 64 * 961, 2 * 64 * 961]
    # NULL and size errors are detected on the host before any device work
    assert lib.wp_hankel_radial(ctypes.byref(p), None, None, 4, None, 0, None, None, None, None) == -1
    ws = ctypes.c_void_p(256)   # never dereferenced: the size check fails first
    assert lib.wp_hankel_radial(ctypes.byref(p), ws, ws, 4, ws, 16, ws, ws, ws, None) == -4
    assert lib.wp_hankel_radial(ctypes.byref(p), ws, ws, 0, ws, 1 << 40, ws, ws, ws, None) == -2
    assert lib.wp_kernelgen_workspace_bytes(ctypes.byref(p), 16) > 0
    assert lib.wp_grid_workspace_bytes(ctypes.byref(p), 16, 1000) > 0
    kern = L.WpWkernels(0, 0, None, None, None, None)
    assert lib.wp_grid(ctypes.byref(p), ctypes.byref(kern), ws, ws, None, 10, ws, 1 << 40, ws, None, None) == -2
    assert lib.wp_dirty_image(ctypes.byref(p), ws, ws, 0.0, ws, None) == -2
    assert lib.wp_strerror(-4) == b"workspace too small or not 256-byte aligned"
    assert lib.wp_version() >= 100
    # the default build keeps no bounds checks
    first = ctypes.c_uint64(7)
    assert lib.wp_bounds_status(ctypes.byref(first), 0) == -8
    # measurement probes: argument errors before any device work
    out = ctypes.c_double()
    assert lib.wp_probe_fp32_fma(0, 8, ws, ctypes.byref(out), None) == -2
    assert lib.wp_probe_fp32_fma(16, 8, None, ctypes.byref(out), None) == -1
    assert lib.wp_probe_l2_taps(None, 1 << 20, 67, 10, 3, ws, ctypes.byref(out), None) == -1
    assert lib.wp_probe_l2_taps(ws, 1 << 20, 0, 10, 3, ws, ctypes.byref(out), None) == -2
    assert lib.wp_probe_l2_taps(ws, 9 * 67 + 32, 67, 10, 3, ws, ctypes.byref(out), None) == -2
    assert lib.wp_probe_l2_taps(ctypes.c_void_p(260), 1 << 20, 67, 10, 3, ws, ctypes.byref(out), None) == -2


def test_projection_route_plan_and_workspace():
    """The projection-slice route is a valid kernelgen value; its workspace holds the
    workspace-pixel n - 1 table and the padded lines (more than the matrix route at a small
    R), and the Hankel adjoint (the matrix route's) refuses it before any device work."""
    L, lib = _lib()
    ps = L.WpPlan(256, 1e-4, 8, 15, 3, 0.01, 512, 0, L.KERNELGEN["projslice"], 0, 0)
    g = L.WpGeometry()
    assert lib.wp_plan_geometry(ctypes.byref(ps), ctypes.byref(g)) == 0
    mx = L.WpPlan(256, 1e-4, 8, 15, 3, 0.01, 512, 0, L.KERNELGEN["tf32x3"], 0, 0)
    assert lib.wp_kernelgen_workspace_bytes(ctypes.byref(ps), 1000) > \
        lib.wp_kernelgen_workspace_bytes(ctypes.byref(mx), 1000) - 3 * 256 * 512 * 4
    ws = ctypes.c_void_p(256)
    assert lib.wp_hankel_adjoint(ctypes.byref(ps), ws, 4, ws, 1 << 40, ws, ws, ws, None) == -8


def test_product_path_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_1904_08463_gb300 import _lib as L

    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(ImportError):
        L.load()


def test_free_kernels_refuses_sets_the_library_did_not_allocate():
    """wp_free_kernels frees only what wp_make_wkernels_owned allocated (flags carries
    WP_KERNELS_OWNED); a caller-owned set and NULL are refused before any CUDA call."""
    L, lib = _lib()
    k = L.WpWkernels(3, 0, None, None, None, None, None, None)
    assert lib.wp_free_kernels(ctypes.byref(k)) == -8
    assert k.P == 3
    assert lib.wp_free_kernels(None) == -1
    out = L.WpWkernels()
    p = L.WpPlan(256, 1e-4, 8, 15, 3, 0.0, 512, 0, 1, 0, 0)
    # no supports with trunc_frac <= 0, and a descending plane list: rejected on the host
    w = (ctypes.c_double * 2)(0.0, 10.0)
    assert lib.wp_make_wkernels_owned(ctypes.byref(p), None, w, 2, None, ctypes.byref(out), None) == -1
    wd = (ctypes.c_double * 2)(10.0, 0.0)
    s = (ctypes.c_int32 * 2)(3, 4)
    assert lib.wp_make_wkernels_owned(ctypes.byref(p), ctypes.c_void_p(16), wd, 2, s, ctypes.byref(out),
                                      None) == -2
    assert out.P == 0 and out.flags == 0


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes views of wp_plan, wp_wkernels and wp_grid_job have the sizes and field offsets
    the C compiler gives the header's structs (checked with gcc, host only)."""
    import ctypes
    import subprocess

    L, _ = _lib()
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "wproj.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(wp_plan), sizeof(wp_wkernels),'
                   ' sizeof(wp_grid_job), offsetof(wp_grid_job, kernels), offsetof(wp_grid_job, V),'
                   ' offsetof(wp_grid_job, stats)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(L.WpPlan), ctypes.sizeof(L.WpWkernels), ctypes.sizeof(L.WpGridJob),
            L.WpGridJob.kernels.offset, L.WpGridJob.V.offset, L.WpGridJob.stats.offset]
    assert got == want


def test_checked_build_compiles_and_exports_the_same_symbols():
    """The -DWP_CHECK_BOUNDS build (index checks on the kernels' main buffer accesses) compiles
    from the same sources and exports every declared function; it is exercised on the GPU by
    tests/test_gpu_bounds.py."""
    from paper_1904_08463_gb300 import build

    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    lib = ctypes.CDLL(build.build_checked())
    for n in _declared():
        assert hasattr(lib, n), n
