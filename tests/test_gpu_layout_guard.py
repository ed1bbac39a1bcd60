"""A kernel set whose offsets do not match its supports (a caller's contract violation) must
not make any kernel read or write outside the plane's block of the cache: the plane is given
the largest support its block holds (or skipped), the other planes are untouched, and the
sentinel after the cache survives.  Every access of these runs stays inside the buffers by
construction (the support is reduced to the block before any index is formed)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _wp():
    import paper_1904_08463_gb300 as wp
    return wp


def _setup(kernelgen="tf32x3"):
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R, os_ = 128, np.deg2rad(4.0) / 128, 256, 4
    plan = wp.Plan(N, dl, os_, 12, 1, 0.0, R, "cubic", kernelgen)
    planes = torch.tensor([0.0, 300.0, 900.0], dtype=torch.float64, device=dev)
    taper = torch.tensor(synth.gaussian_taper_samples(N, dl, R), dtype=torch.float32, device=dev)
    ws = wp.kernelgen_prepare(plan, 3)
    radial, spline_m, _ = wp.hankel_radial(plan, taper, planes, ws)
    return wp, dev, plan, planes, radial, spline_m


def _cache(wp, plan, radial, spline_m, sup_used, off_host, dev, pad=4096):
    """Resample into a buffer with a sentinel tail; returns (cache view, tail)."""
    n = int(off_host[-1])
    big = torch.full((n + pad,), complex(7.0, -7.0), dtype=torch.complex64, device=dev)
    sup = torch.tensor(sup_used, dtype=torch.int32, device=dev)
    off = torch.tensor(off_host, dtype=torch.int64, device=dev)
    wp.resample(plan, radial, spline_m, sup, off, big[:n])
    torch.cuda.synchronize()
    return big[:n], big[n:], sup, off


def test_resample_with_a_block_too_small_stays_inside_it():
    wp, dev, plan, planes, radial, spline_m = _setup()
    good = wp.kernel_layout(plan, [5, 6, 8])          # plane 1 laid out for support 6
    ref, _, _, _ = _cache(wp, plan, radial, spline_m, [5, 6, 8], good, dev)
    bad, tail, _, _ = _cache(wp, plan, radial, spline_m, [5, 10, 8], good, dev)   # claims 10
    assert torch.all(tail == complex(7.0, -7.0))
    a, b = ref.cpu().numpy(), bad.cpu().numpy()
    # every plane, including the violating one (reduced to support 6, the largest that fits),
    # equals the consistent run bit for bit
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_resample_skips_a_plane_with_an_empty_block():
    wp, dev, plan, planes, radial, spline_m = _setup()
    lay = wp.kernel_layout(plan, [5, 6, 8])
    b0, b2 = lay[1] - lay[0], lay[3] - lay[2]
    off = [0, b0, b0, b0 + b2]                          # plane 1: no room at all
    ref, _, _, _ = _cache(wp, plan, radial, spline_m, [5, 6, 8], lay, dev)
    got, tail, _, _ = _cache(wp, plan, radial, spline_m, [5, 6, 8], off, dev)
    assert torch.all(tail == complex(7.0, -7.0))
    r, g = ref.cpu().numpy(), got.cpu().numpy()
    assert np.array_equal(g[:b0].view(np.uint64), r[:b0].view(np.uint64))
    assert np.array_equal(g[b0:].view(np.uint64), r[lay[2]:].view(np.uint64))


@pytest.mark.parametrize("grid_method", [0, 1, 2, 3])
def test_gridding_and_degridding_with_a_block_too_small(grid_method):
    """Gridding and degridding read the violating plane with the support its block holds:
    the grid equals the one made with the consistent layout (visibilities kept away from the
    edges, so that no drop decision depends on the support), and the sentinel survives."""
    wp, dev, plan, planes, radial, spline_m = _setup()
    plan = plan.replace(grid_method=grid_method, grid_tile=32)
    good = wp.kernel_layout(plan, [5, 6, 8])
    c_ok, _, s_ok, o_ok = _cache(wp, plan, radial, spline_m, [5, 6, 8], good, dev)
    c_bad, tail, s_bad, o_bad = _cache(wp, plan, radial, spline_m, [5, 10, 8], good, dev)
    wk_ok = wp.WKernels(planes, s_ok, o_ok, c_ok, radial, spline_m)
    wk_bad = wp.WKernels(planes, s_bad, o_bad, c_bad, radial, spline_m)
    rng = np.random.default_rng(4)
    V = 3000
    du = plan.geometry().du
    uvw = np.stack([rng.uniform(-40, 40, V) * du, rng.uniform(-40, 40, V) * du,
                    rng.uniform(-1000, 1000, V)], 1).astype(np.float32)
    vis = (rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64)
    u_d = torch.tensor(uvw, device=dev).reshape(-1)
    v_d = torch.tensor(vis, device=dev)
    G_ok, st_ok = wp.grid(plan, wk_ok, u_d, v_d)
    G_bad, st_bad = wp.grid(plan, wk_bad, u_d, v_d)
    torch.cuda.synchronize()
    assert torch.all(tail == complex(7.0, -7.0))
    assert st_ok[1].item() == 0 and st_bad[1].item() == 0
    a, b = G_ok.cpu().numpy(), G_bad.cpu().numpy()
    assert np.isfinite(b).all()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
    X = (rng.normal(size=(plan.image_size,) * 2) + 1j * rng.normal(size=(plan.image_size,) * 2)).astype(np.complex64)
    X_d = torch.tensor(X, device=dev)
    d_ok = wp.degrid(plan, wk_ok, u_d, X_d).cpu().numpy()
    d_bad = wp.degrid(plan, wk_bad, u_d, X_d).cpu().numpy()
    assert np.array_equal(d_ok.view(np.uint64), d_bad.view(np.uint64))
