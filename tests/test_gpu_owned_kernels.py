"""Library-owned kernel sets (wp_make_wkernels_owned / wp_free_kernels): the same kernels as
the caller-owned route, bit for bit, with supports from the truncation rule or given; usable
by gridding; freed once."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _bits(t):
    return t.contiguous().cpu().numpy().view(np.uint8)


@pytest.mark.parametrize("trunc,interp", [(0.01, "cubic"), (0.0, "cubic"), (0.01, "linear")])
def test_owned_kernels_equal_caller_owned_and_grid_alike(trunc, interp):
    import ctypes

    import paper_1904_08463_gb300 as wp

    dev = torch.device("cuda")
    N, dl, R = 256, np.deg2rad(2.0) / 256, 512
    planes = np.linspace(0.0, 500.0, 16)
    sup = np.arange(3, 19) if trunc == 0.0 else None
    plan = wp.Plan(N, dl, 8, 18, 3, trunc, R, interp, "bf16x3")
    taper = torch.tensor(synth.gaussian_taper_samples(N, dl, R), dtype=torch.float32, device=dev)
    ref = wp.make_wkernels(plan, taper, planes, supports=sup)
    own = wp.make_wkernels_owned(plan, taper, planes, supports=sup)
    kc = own.c()
    assert kc.P == 16 and kc.flags != 0
    P, n = 16, int(ref.offsets[-1].item())
    lib_sup = torch.empty(P, dtype=torch.int32, device=dev)
    lib_off = torch.empty(P + 1, dtype=torch.int64, device=dev)
    lib_cache = torch.empty(n, dtype=torch.complex64, device=dev)
    cudart = ctypes.CDLL("libcudart.so")
    for dst, src, nbytes in ((lib_sup, kc.support, 4 * P), (lib_off, kc.offsets, 8 * (P + 1)),
                             (lib_cache, kc.cache, 8 * n)):
        assert cudart.cudaMemcpy(ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src), ctypes.c_size_t(nbytes),
                                 3) == 0
    assert np.array_equal(_bits(lib_sup), _bits(ref.support))
    assert np.array_equal(_bits(lib_off), _bits(ref.offsets))
    assert np.array_equal(_bits(lib_cache), _bits(ref.cache))
    assert (kc.spline_m is None) == (interp == "linear")
    # gridding reads both sets alike
    rng = np.random.default_rng(2)
    V = 3000
    du = plan.geometry().du
    uvw = np.stack([rng.uniform(-90, 90, V) * du, rng.uniform(-90, 90, V) * du,
                    rng.uniform(-500, 500, V)], 1).astype(np.float32)
    vis = torch.tensor((rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64), device=dev)
    u_d = torch.tensor(uvw, device=dev).reshape(-1)
    fixed = plan.replace(trunc_frac=0.0, grid_method=0)
    G1, _ = wp.grid(fixed, ref, u_d, vis)
    G2, _ = wp.grid(fixed, own, u_d, vis)
    # same kernels (bitwise above); the grid's cells are flushed with atomics from several
    # planes' items, whose order may differ between two runs
    a, b = G1.cpu().numpy(), G2.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
    own.free()
    assert own._kc.flags == 0 and own._kc.P == 0
    with pytest.raises(RuntimeError):
        own.c()
    own.free()   # a second free is a no-op
