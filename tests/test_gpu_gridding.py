"""GPU parity of binning, gridding, degridding and the dirty image against the oracle."""
import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import IMAGE_TOL, f32, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wp():
    import paper_1904_08463_gb300 as wp

    return wp


def _setup(N, dl, os_, s_max, R, planes, supports, sigma=0.3, grid_tile=0, grid_method=0):
    wp = _wp()
    dev = torch.device("cuda")
    plan = wp.Plan(N, dl, os_, s_max, 1, 0.0, R, "cubic", "fp32", grid_tile, grid_method)
    g = o.Geometry(N, dl, os_, s_max, 1, 0.0, R)
    taper = synth.gaussian_taper_samples(N, dl, R, sigma)
    tap_d = torch.tensor(taper, dtype=torch.float32, device=dev)
    wk = wp.make_wkernels(plan, tap_d, planes, supports=supports)
    ks = o.wkernels(g, f32(taper), planes, supports=supports)
    return wp, dev, plan, g, taper, tap_d, wk, ks


def test_small_imaging_grid_and_dirty_image():
    """20k visibilities, 5 point sources, 16 planes; grid vs oracle grid, and the dirty
    image vs the oracle's dirty image inside the circle (<= 1e-4 of the peak)."""
    d = synth.small_imaging()
    N, dl = d["N"], d["cell_size"]
    planes = np.linspace(0.0, 500.0, 16)
    sup = np.full(16, 5)
    wp, dev, plan, g, taper, tap_d, wk, ks = _setup(N, dl, 8, 15, 512, planes, sup)
    uvw, vis = d["uvw"], d["vis"]
    G, stats = wp.grid(plan, wk, torch.tensor(uvw, device=dev), torch.tensor(vis, device=dev),
                       torch.tensor(d["weight"], device=dev))
    Gh = G.cpu().numpy()
    b = o.bin_vis(g, uvw, planes, sup)
    Go = o.grid(g, ks, b, vis, d["weight"])
    assert np.abs(Gh - Go).max() < 1e-5 * np.abs(Go).max()
    st = stats.cpu().numpy()
    assert st[1] == (b.drop != 0).sum()
    assert st[0] == pytest.approx(float(d["weight"][b.drop == 0].sum()))
    img = wp.dirty_image(plan, tap_d, G, float(st[0])).cpu().numpy()
    ref = o.dirty_image(g, Go, f32(taper), float(st[0]))
    assert np.abs(img - ref).max() < IMAGE_TOL * np.abs(ref).max()
    assert np.all(img[~o.disc_mask(g)] == 0)


@pytest.mark.parametrize("grid_method", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("grid_tile", [32, 64])
@pytest.mark.parametrize("V,seed", [(0, 1), (1, 2), (37, 3), (5000, 4)])
def test_grid_edges_and_conjugation(V, seed, grid_tile, grid_method):
    """Empty input, one visibility, ragged counts; visibilities on and past the grid edge
    (dropped), negative w (conjugated kernels), a plane count off every tile size."""
    N, dl = 96, np.deg2rad(3.0) / 96
    planes = np.array([0.0, 40.0, 130.0, 300.0, 800.0])
    sup = np.array([1, 3, 6, 9, 12])
    wp, dev, plan, g, taper, tap_d, wk, ks = _setup(N, dl, 4, 12, 128, planes, sup, grid_tile=grid_tile,
                                                    grid_method=grid_method)
    rng = np.random.default_rng(seed)
    du = g.du
    uvw = np.stack([rng.uniform(-N / 2 - 2, N / 2 + 2, V) * du, rng.uniform(-N / 2 - 2, N / 2 + 2, V) * du,
                    rng.uniform(-900, 900, V)], 1).astype(np.float32).reshape(V, 3)
    vis = (rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64)
    wt = rng.uniform(0.5, 2.0, V).astype(np.float32)
    G, stats = wp.grid(plan, wk, torch.tensor(uvw, device=dev).reshape(-1), torch.tensor(vis, device=dev),
                       torch.tensor(wt, device=dev))
    b = o.bin_vis(g, uvw, planes, sup)
    Go = o.grid(g, ks, b, vis, wt)
    scale = max(np.abs(Go).max(), 1e-30)
    assert np.abs(G.cpu().numpy() - Go).max() <= 1e-5 * scale
    assert stats[1].item() == (b.drop != 0).sum()
    # degridding of a random grid
    X = (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))).astype(np.complex64)
    Vd = wp.degrid(plan, wk, torch.tensor(uvw, device=dev).reshape(-1), torch.tensor(X, device=dev))
    Vo = o.degrid(g, ks, b, X.astype(np.complex128))
    if V:
        assert np.abs(Vd.cpu().numpy() - Vo).max() <= 2e-5 * max(np.abs(Vo).max(), 1e-30)


@pytest.mark.parametrize("grid_method", [0, 9])
def test_grid_degrid_adjoint_on_gpu(grid_method):
    """<grid(V), X> = <V, degrid(X)> for the GPU operators (unit weights)."""
    N, dl = 128, np.deg2rad(4.0) / 128
    planes = np.linspace(0, 1000, 9)
    sup = np.arange(2, 11)
    wp, dev, plan, g, taper, tap_d, wk, ks = _setup(N, dl, 8, 12, 256, planes, sup, grid_method=grid_method)
    rng = np.random.default_rng(9)
    V = 20000
    uvw = synth.uniform_disc_uvw(V, (N / 2 - 14) * g.du, 1000.0, 10)
    vis = (rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64)
    X = (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))).astype(np.complex64)
    u_d = torch.tensor(uvw, device=dev).reshape(-1)
    G, _ = wp.grid(plan, wk, u_d, torch.tensor(vis, device=dev))
    Vd = wp.degrid(plan, wk, u_d, torch.tensor(X, device=dev))
    lhs = np.vdot(G.cpu().numpy().astype(np.complex128), X.astype(np.complex128))
    rhs = np.vdot(vis.astype(np.complex128), Vd.cpu().numpy().astype(np.complex128))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


def test_dirty_image_and_adjoint_on_synthetic_grids():
    """The image stage alone on seeded synthetic grids (sizes 64 and 1024): vs the oracle's
    numpy transform, and image_to_grid as the adjoint of the linear part of dirty_image."""
    wp = _wp()
    dev = torch.device("cuda")
    for N, seed in ((64, 1), (1024, 2)):
        dl = np.deg2rad(4.0) / N
        R = 512
        plan = wp.Plan(N, dl, 8, 15, 3, 0.01, R)
        g = o.Geometry(N, dl, 8, 15, 3, 0.01, R)
        taper = synth.gaussian_taper_samples(N, dl, R, 0.25)
        rng = np.random.default_rng(seed)
        X = (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))).astype(np.complex64)
        tap_d = torch.tensor(taper, dtype=torch.float32, device=dev)
        img = wp.dirty_image(plan, tap_d, torch.tensor(X, device=dev), 3.5).cpu().numpy()
        ref = o.dirty_image(g, X.astype(np.complex128), f32(taper), 3.5)
        assert np.abs(img - ref).max() < 1e-5 * np.abs(ref).max()
        Y = rng.normal(size=(N, N)).astype(np.float32)
        Gy = wp.image_to_grid(plan, tap_d, torch.tensor(Y, device=dev), 3.5).cpu().numpy().astype(np.complex128)
        # <Re A X, Y> = Re <X, A^H Y>
        lhs = float(np.sum(ref * Y))
        rhs = float(np.real(np.vdot(Gy, X.astype(np.complex128))))
        assert abs(lhs - rhs) < 1e-4 * abs(lhs) + 1e-6


@pytest.mark.parametrize("V,P,seed", [(20000, 16, 1), (1001, 7, 2), (64, 64, 3), (5, 1, 4)])
def test_plane_values_are_means_of_equal_count_chunks(V, P, seed):
    """Alg. 2 steps 1-3: sort |w|, P equal-count chunks (first V mod P one longer), means."""
    wp = _wp()
    uvw = synth.uniform_disc_uvw(V, 1000.0, 700.0, seed)
    got = wp.plane_values(torch.tensor(uvw, device="cuda").reshape(-1), P).cpu().numpy()
    ref = o.mean_w_planes(uvw[:, 2].astype(np.float64), P)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)
    assert np.all(np.diff(got) >= 0)


@pytest.mark.parametrize("grid_method", [0, 3, 5, 6, 7, 8, 9])
def test_non_finite_coordinates_are_dropped(grid_method):
    """NaN / infinite u, v or w: the GPU binning drops and counts them as the oracle does, the
    grid of the rest is unchanged, degridding returns 0 for them, and the plane values are the
    chunk means of the finite |w| only."""
    N, dl = 96, np.deg2rad(3.0) / 96
    planes = np.array([0.0, 40.0, 130.0, 300.0, 800.0])
    sup = np.array([1, 3, 6, 9, 12])
    wp, dev, plan, g, taper, tap_d, wk, ks = _setup(N, dl, 4, 12, 128, planes, sup, grid_method=grid_method)
    rng = np.random.default_rng(9)
    V = 2000
    du = g.du
    uvw = np.stack([rng.uniform(-30, 30, V) * du, rng.uniform(-30, 30, V) * du,
                    rng.uniform(-900, 900, V)], 1).astype(np.float32)
    bad = rng.choice(V, 60, replace=False)
    vals = np.array([np.nan, np.inf, -np.inf], dtype=np.float32)
    uvw[bad, rng.integers(0, 3, 60)] = vals[rng.integers(0, 3, 60)]
    vis = (rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64)
    u_d = torch.tensor(uvw, device=dev).reshape(-1)
    G, stats = wp.grid(plan, wk, u_d, torch.tensor(vis, device=dev))
    b = o.bin_vis(g, uvw, planes, sup)
    assert (b.drop[bad] == 1).all()
    assert stats[1].item() == (b.drop != 0).sum()
    Go = o.grid(g, ks, b, vis)
    assert np.abs(G.cpu().numpy() - Go).max() <= 1e-5 * np.abs(Go).max()
    X = (rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))).astype(np.complex64)
    Vd = wp.degrid(plan, wk, u_d, torch.tensor(X, device=dev)).cpu().numpy()
    assert np.all(Vd[bad] == 0)
    pv = wp.plane_values(u_d, 7).cpu().numpy()
    assert np.allclose(pv, o.mean_w_planes(uvw[:, 2].astype(np.float64), 7), rtol=1e-13, atol=0)
    assert np.all(np.isfinite(pv)) and np.all(np.diff(pv) >= 0)


@pytest.mark.parametrize("interp", ["cubic", "linear"])
def test_on_the_fly_taps_need_no_cache_and_match_the_cache_gridder(interp):
    """grid_method 4 interpolates every tap from the plane's radial line in shared memory with
    the resample's own evaluation: with the cache pointer left NULL it grids the same values as
    the cache-reading method 3 (to FP32 accumulation order) and as the oracle."""
    import paper_1904_08463_gb300 as wp

    dev = torch.device("cuda")
    N, dl = 128, np.deg2rad(3.0) / 128
    planes = np.array([0.0, 90.0, 260.0, 700.0])
    sup = np.array([2, 5, 9, 14])
    plan = wp.Plan(N, dl, 8, 14, 1, 0.0, 256, interp, "fp32", 64, 3)
    taper = synth.gaussian_taper_samples(N, dl, 256)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), planes, supports=sup)
    rng = np.random.default_rng(11)
    V = 3000
    uvw = np.stack([rng.uniform(-N / 2 + 16, N / 2 - 16, V) / (N * dl), rng.uniform(-N / 2 + 16, N / 2 - 16, V) / (N * dl),
                    rng.uniform(-800, 800, V)], 1).astype(np.float32)
    vis = (rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64)
    u_d, v_d = torch.tensor(uvw, device=dev).reshape(-1), torch.tensor(vis, device=dev)
    G3, _ = wp.grid(plan, wk, u_d, v_d)
    wk_nocache = wp.WKernels(wk.w_planes, wk.support, wk.offsets, None, wk.radial, wk.spline_m)
    G4, _ = wp.grid(plan.replace(grid_method=4), wk_nocache, u_d, v_d)
    G3, G4 = G3.cpu().numpy(), G4.cpu().numpy()
    assert np.abs(G4 - G3).max() <= 2e-6 * np.abs(G3).max()
    g = o.Geometry(N, dl, 8, 14, 1, 0.0, 256, 0 if interp == "cubic" else 1)
    ks = o.wkernels(g, f32(taper), planes, supports=sup)
    b = o.bin_vis(g, uvw, planes, sup)
    Go = o.grid(g, ks, b, vis.astype(np.complex128))
    assert rel_l2(G4, Go) < 1e-5


@pytest.mark.parametrize("grid_method,grid_tile", [(5, 32), (5, 64), (6, 32), (6, 64), (9, 64)])
def test_plane_groups_with_a_ragged_last_group(grid_method, grid_tile):
    """19 planes -- two full groups of 8 and a ragged group of 3 -- with supports 2..38, so that
    footprints reach up to two tiles away: the plane-group gridders against the oracle, with
    weights and both signs of w."""
    N, dl = 256, np.deg2rad(4.0) / 256
    planes = np.linspace(0.0, 1800.0, 19)
    sup = np.linspace(2, 38, 19).round().astype(int)
    wp, dev, plan, g, taper, tap_d, wk, ks = _setup(N, dl, 4, 38, 256, planes, sup, grid_tile=grid_tile,
                                                    grid_method=grid_method)
    rng = np.random.default_rng(23)
    V = 6000
    uvw = np.stack([rng.uniform(-N / 2, N / 2, V) * g.du, rng.uniform(-N / 2, N / 2, V) * g.du,
                    rng.uniform(-1900, 1900, V)], 1).astype(np.float32)
    vis = (rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64)
    wt = rng.uniform(0.5, 2.0, V).astype(np.float32)
    G, stats = wp.grid(plan, wk, torch.tensor(uvw, device=dev).reshape(-1), torch.tensor(vis, device=dev),
                       torch.tensor(wt, device=dev))
    b = o.bin_vis(g, uvw, planes, sup)
    Go = o.grid(g, ks, b, vis, wt)
    assert np.abs(G.cpu().numpy() - Go).max() <= 1e-5 * np.abs(Go).max()
    assert stats[1].item() == (b.drop != 0).sum() > 0
