"""Allocation-free gridding (wp_grid_static) against the ordinary entry point (wp_grid).

wp_grid_static exists for callers that cannot allocate device memory (pipelines that
reserve all GPU memory up front, plug-ins that may only use memory they are handed): it
takes its scratch from an array compiled into the library instead of a caller workspace.
This file is collected last on purpose, so that a run stopping at the first failure has
already run every other test; it also passes when run on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _setup():
    import paper_1904_08463_gb300 as wp

    dev = torch.device("cuda")
    d = synth.small_imaging(seed=21)
    N, dl = d["N"], d["cell_size"]
    plan = wp.Plan(N, dl, 8, 15, 3, 0.0, 512, "cubic", "fp32")
    taper = torch.tensor(synth.gaussian_taper_samples(N, dl, 512), dtype=torch.float32, device=dev)
    planes = np.linspace(0.0, 500.0, 16)
    wk = wp.make_wkernels(plan, taper, planes, supports=np.full(16, 5))
    uvw = torch.tensor(d["uvw"], device=dev).reshape(-1)
    vis = torch.tensor(d["vis"], device=dev)
    wt = torch.tensor(np.linspace(0.5, 1.5, vis.numel()).astype(np.float32), device=dev)
    return wp, plan, wk, uvw, vis, wt


def _call_static(lib, plan, wk, uvw, vis, wt, V, grid, stats):
    kc = wk.c()
    return lib.wp_grid_static(ctypes.byref(plan.c()), ctypes.byref(kc), ctypes.c_void_p(uvw.data_ptr()),
                              ctypes.c_void_p(vis.data_ptr()), ctypes.c_void_p(wt.data_ptr()), V,
                              ctypes.c_void_p(grid.data_ptr()), ctypes.c_void_p(stats.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_scratch_gridding_matches_workspace_gridding_twice():
    from paper_1904_08463_gb300 import _lib

    wp, plan, wk, uvw, vis, wt = _setup()
    lib = _lib.load()
    V = vis.numel()
    ref, ref_stats = wp.grid(plan, wk, uvw, vis, wt)
    torch.cuda.synchronize()
    R = ref.cpu().numpy()
    outs = [(torch.zeros_like(ref), torch.zeros(2, dtype=torch.float64, device=vis.device)) for _ in range(2)]
    # set-up call (V = 0: looks up the array, which commits it on this device, grids nothing)
    assert _call_static(lib, plan, wk, uvw, vis, wt, 0, outs[0][0], outs[0][1]) == 0
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for G, stats in outs:   # two calls in a row: the shared scratch must not leak between calls
        assert _call_static(lib, plan, wk, uvw, vis, wt, V, G, stats) == 0
        torch.cuda.synchronize()
        # nothing allocated on the device by the calls, through torch or the driver
        assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
        assert np.abs(G.cpu().numpy() - R).max() <= 1e-5 * np.abs(R).max()
        assert np.allclose(stats.cpu().numpy(), ref_stats.cpu().numpy(), rtol=1e-12)


def test_static_scratch_rejects_oversize_problem_before_launch():
    from paper_1904_08463_gb300 import _lib

    wp, plan, wk, uvw, vis, wt = _setup()
    lib = _lib.load()
    G = torch.zeros((plan.image_size, plan.image_size), dtype=torch.complex64, device=vis.device)
    stats = torch.zeros(2, dtype=torch.float64, device=vis.device)
    # 10^8 visibilities need far more than the static scratch: refused, nothing read
    assert _call_static(lib, plan, wk, uvw, vis, wt, 100_000_000, G, stats) == -2
    torch.cuda.synchronize()
    assert float(torch.abs(G).max()) == 0.0
