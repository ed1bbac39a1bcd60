"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle routine to something other than itself: a library routine,
a closed form, a table printed in a book or in the paper, an invariant, or brute force.
They are chosen so that a plausible slip (a dropped 2 pi, r_i = i dr instead of
(i + 1/2) dr, a sign flip of the w-screen, a transposed tap index, a wrong spline end
condition, an off-by-one in the oversampling offset) fails at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.special as sp
from scipy.interpolate import CubicSpline

import synth
from oracle import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


# ----------------------------------------------------------------------------- J0
def test_j0_matches_library():
    x = np.concatenate([np.linspace(0.0, 50.0, 2001), np.linspace(50.0, 1200.0, 3001)])
    assert np.abs(o.j0(x) - sp.j0(x)).max() < 3e-14


def test_j0_table_zeros_and_origin():
    z = _golden("j0_zeros.txt")[:, 1]
    assert np.abs(o.j0(z)).max() < 2e-15 * 10
    assert o.j0(np.array([0.0]))[0] == pytest.approx(1.0, abs=1e-15)
    # J0 changes sign across each zero
    assert np.all(o.j0(z - 1e-6) * o.j0(z + 1e-6) < 0)


# ---------------------------------------------------------------------- Hankel (Eq. 12)
def test_hankel_gaussian_closed_form():
    """exp(-a r^2) <-> (pi/a) exp(-pi^2 rho^2 / a); the midpoint rule's leading error is the
    Euler-Maclaurin term (h^2/24)(g'(0) - g'(r_max)) = pi h^2 / 12 for g = 2 pi r f J0."""
    r_max, a = 1.0, 40.0
    rho = np.linspace(0.0, 3.0, 31)
    G = np.pi / a * np.exp(-np.pi ** 2 * rho ** 2 / a)
    errs = []
    for R in (256, 512):
        r = (np.arange(R) + 0.5) * r_max / R
        M = o.hankel(np.exp(-a * r * r), r_max, rho)
        h = r_max / R
        assert np.abs(M.imag).max() == 0.0
        assert np.abs(M - G - np.pi * h * h / 12).max() < 1.5e-9 * (256 / R) ** 4
        errs.append(np.abs(M - G).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=2e-3)


def test_hankel_disc_is_jinc():
    """Disc of radius b <-> b J1(2 pi b rho) / rho (jinc), with the midpoint-rule
    Euler-Maclaurin term (h^2/24)(g'(0) - g'(b)), g(r) = 2 pi r J0(2 pi rho r)."""
    b = 1.0
    rho = np.linspace(0.05, 5.0, 40)
    G = b * sp.j1(2 * np.pi * b * rho) / rho
    for R in (256, 512):
        h = b / R
        M = o.hankel(np.ones(R), b, rho).real
        gpb = 2 * np.pi * (sp.j0(2 * np.pi * rho * b) - 2 * np.pi * rho * b * sp.j1(2 * np.pi * rho * b))
        corr = -(h * h / 24) * (gpb - 2 * np.pi)
        assert np.abs(M - G - corr).max() < 1e-8 * (256 / R) ** 4
    # rho = 0: area of the disc
    assert o.hankel(np.ones(2048), b, np.array([0.0]))[0].real == pytest.approx(np.pi * b * b, rel=1e-6)


def test_hankel_matrix_equals_direct():
    R, r_max = 300, 0.7
    rho = np.linspace(0, 40, 17)
    rng = np.random.default_rng(0)
    f = rng.normal(size=R) + 1j * rng.normal(size=R)
    H = o.hankel_matrix(R, r_max, rho)
    assert np.allclose(o.hankel_apply(H, f), o.hankel(f, r_max, rho), rtol=0, atol=1e-13)


# ------------------------------------------------------- w-screen x taper -> radial kernel
def _paraxial_geometry(R):
    N, r_max = 64, 0.02
    g = o.Geometry(N, 2 * r_max / N, 8, 15, 3, 0.01, R)
    a = 40.0 / r_max ** 2
    return g, a, np.exp(-a * g.r_nodes() ** 2)


@pytest.mark.parametrize("w", [0.0, 2000.0, 20000.0])
def test_radial_kernel_complex_gaussian(w):
    """Narrow Gaussian taper times the w-screen: for r << 1 the screen is the paraxial chirp
    exp(-j pi w r^2), so the kernel is du^2 (pi/c) exp(-pi^2 rho^2 / c), c = a + j pi w.
    The quartic term of sqrt(1-r^2) contributes < 3e-6 here.  A conjugated screen (wrong
    gridding sign) is off by ~0.1-1 and fails."""
    g, a, tap = _paraxial_geometry(512)
    C = o.radial_kernel(g, tap, w)
    c = a + 1j * np.pi * w
    G = g.du ** 2 * np.pi / c * np.exp(-np.pi ** 2 * g.rho() ** 2 / c)
    h = g.r_max / g.radial_samples
    em = g.du ** 2 * np.pi * h * h / 12
    scale = np.abs(G).max()
    assert np.abs(C - G - em).max() / scale < 1e-5
    if w:
        assert np.abs(C - np.conj(G)).max() / scale > 0.05


def test_w0_kernel_is_transformed_taper():
    g = o.Geometry(256, np.deg2rad(2) / 256, 8, 15, 3, 0.01, 512)
    tap = o.gaussian_taper(g)
    C0 = o.radial_kernel(g, tap, 0.0)
    direct = o.hankel(tap.astype(np.complex128), g.r_max, g.rho()) * g.du ** 2
    assert np.abs(C0 - direct).max() < 1e-15
    assert np.abs(C0.imag).max() == 0.0


def test_negative_w_is_conjugate():
    """Section 4.1: the kernel of -w is the conjugate of the kernel of +w."""
    g = o.Geometry(256, np.deg2rad(2) / 256, 8, 15, 3, 0.01, 512)
    tap = o.gaussian_taper(g)
    for w in (37.0, 480.0):
        assert np.abs(o.radial_kernel(g, tap, -w) - np.conj(o.radial_kernel(g, tap, w))).max() < 1e-17


# ------------------------------------------------------------------------------ spline
def test_spline_matches_scipy_clamped_natural():
    rng = np.random.default_rng(1)
    K = 97
    y = rng.normal(size=K) + 1j * rng.normal(size=K)
    m = o.spline_m(y)
    x = np.linspace(0, K - 1, 5000)
    ours = o.spline_eval(y, m, x)
    ref = CubicSpline(np.arange(K), y, bc_type=((1, 0.0), (2, 0.0)))(x)
    assert np.abs(ours - ref).max() < 1e-12
    lin = o.spline_eval(y, m, x, interp=1)
    assert np.abs(lin - np.interp(x, np.arange(K), y.real) - 1j * np.interp(x, np.arange(K), y.imag)).max() < 1e-14


def test_spline_reproduces_admissible_cubic():
    """A cubic with zero slope at 0 and zero curvature at the last node is reproduced."""
    K = 64
    xe = K - 1.0
    f = lambda x: 1.0 + 1e-4 * (x ** 3 - 3 * xe * x ** 2) * (1 + 0.5j)
    y = f(np.arange(K, dtype=np.float64))
    m = o.spline_m(y)
    x = np.linspace(0, xe, 777)
    assert np.abs(o.spline_eval(y, m, x) - f(x)).max() < 1e-9 * np.abs(y).max()


# -------------------------------------------------------------------- 2D kernel cache
def _small_imaging_geometry(R=512):
    return o.Geometry(256, np.deg2rad(2.0) / 256, 8, 15, 3, 0.01, R)


def test_resample_matches_direct_transform_at_tap_radius():
    """Every tap equals the Hankel transform evaluated directly at the tap's exact radius,
    up to the cubic-spline error; taps beyond the support radius are zero."""
    g = _small_imaging_geometry()
    tap = o.gaussian_taper(g)
    w, S = 450.0, 6
    C = o.radial_kernel(g, tap, w)
    cache = o.resample(g, C, S)
    os_ = g.oversampling
    jj = np.arange(2 * S + 1) - S
    fv, fu, jy, jx = np.meshgrid(np.arange(os_), np.arange(os_), jj, jj, indexing="ij")
    q = (os_ * jx - fu) ** 2 + (os_ * jy - fv) ** 2
    inside = q <= (os_ * S) ** 2
    assert np.all(cache[~inside] == 0)
    # direct transform at a subsample of exact radii
    idx = np.flatnonzero(inside.ravel())[:: 37]
    rho = np.sqrt(q.ravel()[idx].astype(np.float64)) * g.du / os_
    direct = o.hankel(o.screen(g, tap, w), g.r_max, rho) * g.du ** 2
    err = np.abs(cache.ravel()[idx] - direct).max() / np.abs(C).max()
    # cubic-spline error (5/384) h^4 |C''''| with the band limit 2 pi r_max of C: <= 3e-4 |C|;
    # the taper here is smooth enough that it is two orders lower
    assert err < 1e-5
    # linear interpolation is measurably worse but bounded (h^2/8 |C''|)
    g_lin = o.Geometry(**{**g.__dict__, "interp": 1})
    lin = o.resample(g_lin, C, S).ravel()[idx]
    e_lin = np.abs(lin - direct).max() / np.abs(C).max()
    assert 10 * err < e_lin < 5e-2


def test_subkernel_symmetry():
    """Radial symmetry: with fu == fv a sub-kernel is symmetric under jx <-> jy; and the
    (fu, fv) sub-kernel is the transpose of the (fv, fu) one."""
    g = _small_imaging_geometry()
    C = o.radial_kernel(g, o.gaussian_taper(g), 300.0)
    k = o.resample(g, C, 5)
    for f in range(g.oversampling):
        assert np.array_equal(k[f, f], k[f, f].T)
    assert np.array_equal(k[2, 5], k[5, 2].T)


def test_truncation_support():
    """Section 3.1: the support is the last radius where |C| >= 1 % of max, in whole cells."""
    g = _small_imaging_geometry()
    C = np.zeros(g.k_out, dtype=np.complex128)
    C[:50] = np.linspace(1.0, 0.0, 50)          # |C[k]| >= 0.01 for k <= 49*0.99 -> k <= 49
    C[49] = 0.0100000001
    assert o.support(g, C) == (49 + 7) // 8
    C[49] = 0.0099999999
    assert o.support(g, C) == (48 + 7) // 8
    C2 = np.zeros(g.k_out, dtype=np.complex128)
    C2[0] = 1.0
    assert o.support(g, C2) == g.min_support
    C3 = np.ones(g.k_out, dtype=np.complex128)
    assert o.support(g, C3) == g.max_support


def test_workspace_sizes_printed_in_paper():
    rows = _golden("workspace_sizes.txt").astype(int)
    for s, ws, fft, full in rows:
        assert o.workspace_size(s) == ws
        assert ws * 8 == fft
        assert 2 * s + 1 == full
    g = o.Geometry(64, 1e-3, 8, 4, 1, 0.01, 64)
    ks = o.wkernels(g, np.ones(64), [0.0], supports=[4])
    assert ks.offsets[1] == 64 * 9 * 9          # 64 kernels per plane at oversampling 8


def test_fft_route_agrees_with_hankel_route():
    """Section 4.3: the order-0 Hankel transform equals the 2D Fourier transform of a radially
    symmetric function.  For a taper that vanishes smoothly inside the disc both routes give
    the same cache to discretisation error (dominated by the FFT route's linear taper
    interpolation, ~1e-6 at R = 4096)."""
    g, a, tap = _paraxial_geometry(4096)
    for w in (0.0, 20000.0):
        hk = o.resample(g, o.radial_kernel(g, tap, w), 10)
        fk = o.fft_wkernel(g, tap, w, 10)
        assert np.linalg.norm(hk - fk) / np.linalg.norm(hk) < 5e-6


def test_projslice_line_is_v0_slice_of_2d_route():
    """Section 4.3.1: the 1D transform of the workspace image projected onto l is the v = 0
    slice of its 2D transform -- exactly, for the discrete transforms.  Sample k of the
    projection route's line is tap (jx, S) of sub-kernel (fu, 0) of the 2D-FFT route with
    os (jx - S) - fu = k, here at w = 0 and at a w whose screen wraps many turns."""
    g = o.Geometry(96, np.deg2rad(3.0) / 96, 4, 12, 1, 0.0, 512)
    tap = o.gaussian_taper(g)
    S, os_ = g.max_support, g.oversampling
    for w in (0.0, 700.0):
        line = o.projslice_radial(g, tap, w)
        full = o.fft_wkernel(g, tap, w, S, circular=False)        # [fv][fu][jy][jx]
        k = np.arange(os_ * S + 1)
        m = -(-k // os_)                                          # ceil(k / os)
        fu = os_ * m - k
        ref = full[0, fu, S, S + m]
        assert np.abs(line[k] - ref).max() < 1e-12 * np.abs(ref).max()


def test_projslice_gaussian_closed_form():
    """A Gaussian taper exp(-r^2 / (2 s^2)) at w = 0 transforms to 2 pi s^2 exp(-2 pi^2 s^2 rho^2);
    with 12.8 workspace pixels per s and the disc edge at 10 s, the projection route's line
    (in tap units, times du^2) matches it to the taper's linear interpolation (~1e-6)."""
    g = o.Geometry(256, np.deg2rad(2.0) / 256, 2, 127, 1, 0.0, 4096)
    s_ = 0.05 * g.fov
    tap = np.exp(-g.r_nodes() ** 2 / (2 * s_ * s_))
    line = o.projslice_radial(g, tap, 0.0)
    rho = g.rho()
    ref = 2 * np.pi * s_ ** 2 * np.exp(-2 * np.pi ** 2 * s_ ** 2 * rho ** 2) * g.du ** 2
    n = 2 * g.oversampling * 10                  # out to 10 uv cells (the kernel is ~1e-30 there)
    assert np.abs(line[:n] - ref[:n]).max() < 2e-6 * ref[0]
    assert np.abs(line[:n].imag).max() < 1e-12 * ref[0]


def test_projslice_route_agrees_with_hankel_route():
    """Both routes approximate the same 2D transform of a radially symmetric function: for a
    taper that vanishes smoothly inside the disc their caches agree to discretisation error."""
    g, a, tap = _paraxial_geometry(4096)
    for w in (0.0, 20000.0):
        hk = o.resample(g, o.radial_kernel(g, tap, w), 10)
        pk = o.resample(g, o.projslice_radial(g, tap, w), 10)
        assert np.linalg.norm(hk - pk) / np.linalg.norm(hk) < 5e-6


# ------------------------------------------------------------------------------ binning
def test_binning_rules():
    N, dl, os_ = 64, 1e-3, 8
    g = o.Geometry(N, dl, os_, 4, 1, 0.01, 64)
    du = g.du
    us = []
    expect = []
    for k, f in [(30, 0), (30, 3), (33, 7), (20, 5)]:
        us.append(((k - N / 2) + f / os_) * du)
        expect.append((k, f))
    uvw = np.array([[u, u, 10.0] for u in us], dtype=np.float32)
    b = o.bin_vis(g, uvw, [0.0, 100.0], [4, 4])
    for i, (k, f) in enumerate(expect):
        # brute force: nearest point of the 1/os lattice to the float32 coordinate
        uc = float(np.float32(us[i])) / du + N / 2
        cands = [(abs(uc - (kk + ff / os_)), kk, ff) for kk in range(N) for ff in range(os_)]
        _, kk, ff = min(cands)
        assert (b.iu[i], b.fu[i]) == (kk, ff) == (k, f)
        assert (b.iv[i], b.fv[i]) == (k, f)
    assert np.all(b.plane == 0) and np.all(b.conj == 0) and np.all(b.drop == 0)


def test_binning_plane_conj_drop():
    N, dl, os_ = 64, 1e-3, 8
    g = o.Geometry(N, dl, os_, 4, 1, 0.01, 64)
    du = g.du
    planes = [0.0, 100.0, 300.0]
    uvw = np.array([[0, 0, 49.0], [0, 0, 50.0], [0, 0, -51.0], [0, 0, 250.0], [0, 0, -1000.0],
                    [(-N / 2 + 3) * du, 0, 0.0], [(-N / 2 + 4) * du, 0, 0.0],
                    [(N / 2 - 5) * du, 0, 0.0], [(N / 2 - 4) * du, 0, 0.0]], dtype=np.float32)
    b = o.bin_vis(g, uvw, planes, [4, 4, 4])
    assert list(b.plane[:5]) == [0, 0, 1, 2, 2]      # tie at 50 -> lower plane
    assert list(b.conj[:5]) == [0, 0, 1, 0, 1]
    assert list(b.drop) == [0, 0, 0, 0, 0, 1, 0, 0, 1]


def test_mean_w_planes_equal_count_chunks():
    w = np.array([-5.0, 1.0, 2.0, -3.0, 4.0, 6.0])
    assert np.allclose(o.mean_w_planes(w, 3), [1.5, 3.5, 5.5])


def test_non_finite_coordinates_are_dropped_and_left_out_of_the_plane_values():
    """No nearest plane or grid cell exists for a NaN or infinite coordinate: such a
    visibility is dropped (and counted) whatever its other coordinates, and its |w| takes no
    part in the plane values; chunks left empty take the largest finite |w|."""
    N, dl, os_ = 64, 1e-3, 8
    g = o.Geometry(N, dl, os_, 4, 1, 0.01, 64)
    nan, inf = np.float32(np.nan), np.float32(np.inf)
    uvw = np.array([[0, 0, 10.0], [nan, 0, 10.0], [0, inf, 10.0], [0, 0, nan], [0, 0, -inf],
                    [0, 0, 150.0]], dtype=np.float32)
    b = o.bin_vis(g, uvw, [0.0, 100.0, 300.0], [4, 4, 4])
    assert list(b.drop) == [0, 1, 1, 1, 1, 0]
    assert list(b.plane[[0, 5]]) == [0, 1]
    w = np.array([-5.0, np.nan, 1.0, 2.0, np.inf, -3.0, 4.0, 6.0, -np.inf])
    assert np.allclose(o.mean_w_planes(w, 3), [1.5, 3.5, 5.5])
    assert np.allclose(o.mean_w_planes(np.array([2.0, np.nan, 7.0]), 4), [2.0, 7.0, 7.0, 7.0])
    assert np.allclose(o.mean_w_planes(np.array([np.nan, np.inf]), 2), [0.0, 0.0])


# ------------------------------------------------------------------- gridding / degridding
def _random_problem(seed=0, V=300):
    g = o.Geometry(64, np.deg2rad(2.0) / 64, 4, 5, 2, 0.01, 128)
    tap = o.gaussian_taper(g)
    planes = np.array([0.0, 120.0, 300.0, 500.0])
    ks = o.wkernels(g, tap, planes, supports=[2, 3, 4, 5])
    rng = np.random.default_rng(seed)
    du = g.du
    uvw = np.stack([rng.uniform(-25, 25, V) * du, rng.uniform(-25, 25, V) * du,
                    rng.uniform(-520, 520, V)], axis=1).astype(np.float32)
    vis = (rng.normal(size=V) + 1j * rng.normal(size=V)).astype(np.complex64)
    return g, tap, ks, o.bin_vis(g, uvw, planes, ks.support), uvw, vis


def test_grid_degrid_adjoint():
    g, tap, ks, b, uvw, vis = _random_problem()
    G = o.grid(g, ks, b, vis)
    rng = np.random.default_rng(5)
    X = rng.normal(size=G.shape) + 1j * rng.normal(size=G.shape)
    lhs = np.vdot(G, X)
    rhs = np.vdot(vis.astype(np.complex128), o.degrid(g, ks, b, X))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_single_visibility_reproduces_subkernel():
    g, tap, ks, _, _, _ = _random_problem()
    du, N, os_ = g.du, g.image_size, g.oversampling
    for w, conj in ((300.0, False), (-300.0, True)):
        uvw = np.array([[(3 + 1 / os_) * du, (-2 + 3 / os_) * du, w]], dtype=np.float32)
        b = o.bin_vis(g, uvw, ks.w_planes, ks.support)
        assert (b.plane[0], b.fu[0], b.fv[0]) == (2, 1, 3)
        G = o.grid(g, ks, b, np.array([1.0 + 0j], dtype=np.complex64))
        S = 4
        sub = ks.cache[ks.offsets[2]:ks.offsets[3]].reshape(os_, os_, 2 * S + 1, 2 * S + 1)[3, 1]
        iu, iv = b.iu[0], b.iv[0]
        win = G[iv - S:iv + S + 1, iu - S:iu + S + 1]
        assert np.array_equal(win, np.conj(sub) if conj else sub)
        assert np.abs(G).sum() == pytest.approx(np.abs(sub).sum())


def test_weights_scale_linearly():
    g, tap, ks, b, uvw, vis = _random_problem(3, 50)
    wt = np.linspace(0.5, 2.0, 50).astype(np.float32)
    G1 = o.grid(g, ks, b, vis, wt)
    G2 = o.grid(g, ks, b, (vis * wt).astype(np.complex64))
    assert np.abs(G1 - G2).max() < 1e-6 * np.abs(G1).max()


# ----------------------------------------------------------------------- dirty image
def _imaging_error(os_, planes_count, seed=7, S_max=15):
    """Max error of the w-projection dirty image against the brute-force direct image
    over the inner 3/4 of the circular region (outside it the division by the taper,
    0.04 at the rim for sigma = 0.2 FOV, magnifies the kernel-truncation error)."""
    N = 64
    dl = np.deg2rad(4.0) / N
    g = o.Geometry(N, dl, os_, S_max, 2, 0.001, 512)
    rng = np.random.default_rng(seed)
    V = 1500
    du = g.du
    rad = (N / 2 - S_max - 2) * du * np.sqrt(rng.random(V))
    th = 2 * np.pi * rng.random(V)
    uvw = np.stack([rad * np.cos(th), rad * np.sin(th), rng.uniform(-400, 400, V)], 1).astype(np.float32)
    sky = synth.sources_in_disc(3, np.deg2rad(1.5), seed + 1, 0.5, 1.0)
    vis = synth.predict(uvw, sky)
    tap = o.gaussian_taper(g, 0.2)
    planes = np.linspace(0, 400, planes_count) if planes_count > 1 else np.array([0.0])
    ks = o.wkernels(g, tap, planes)
    b = o.bin_vis(g, uvw, planes, ks.support)
    keep = b.drop == 0
    assert keep.all()
    img = o.dirty_image(g, o.grid(g, ks, b, vis), tap, float(keep.sum()))
    im_, il_ = np.nonzero(o.disc_mask(g))
    inner = np.hypot(il_ - N / 2, im_ - N / 2) < 0.75 * N / 2
    im_, il_ = im_[inner], il_[inner]
    ref = o.dft_image(g, uvw, vis, pixels=(il_, im_))
    return np.abs(img[im_, il_] - ref).max() / np.abs(ref).max()


def test_dirty_image_matches_brute_force_direct_imaging():
    """Eq. 2 adjoint evaluated pixel by pixel vs the w-projection dirty image.  The gap is
    the method's own error (oversampling, w-plane quantisation, kernel truncation), so it
    must shrink when oversampling is raised and grow without w-correction."""
    e8 = _imaging_error(8, 17)
    assert e8 < 1.2e-2
    e2 = _imaging_error(2, 17)
    assert e2 > 3 * e8                 # coarser oversampling -> further from the direct sum
    e_off = _imaging_error(8, 1)       # no w-correction (single plane at w = 0)
    assert e_off > 5 * e8


def test_point_source_at_phase_centre_peak_equals_flux():
    N = 64
    g = o.Geometry(N, np.deg2rad(2.0) / N, 8, 15, 2, 0.001, 256)
    uvw = synth.uniform_disc_uvw(800, (N / 2 - 17) * g.du, 300.0, 11)
    vis = np.full(800, 0.7 + 0j, dtype=np.complex64)
    tap = o.gaussian_taper(g, 0.2)
    planes = np.linspace(0, 300, 8)
    ks = o.wkernels(g, tap, planes)
    b = o.bin_vis(g, uvw, planes, ks.support)
    img = o.dirty_image(g, o.grid(g, ks, b, vis), tap, float((b.drop == 0).sum()))
    # the gridded kernel sums to t(0) = 1 up to the 0.1 % truncation -> peak = flux
    assert img[N // 2, N // 2] == pytest.approx(0.7, rel=3e-3)
    assert img.max() == img[N // 2, N // 2]


def test_cellwise_gridding_equals_full_oracle_grid():
    """The cell-by-cell form (taps evaluated from the radial lines) reproduces the full
    oracle grid exactly at every sampled cell, conjugated kernels included."""
    g, tap, ks, b, uvw, vis = _random_problem(1, 400)
    G = o.grid(g, ks, b, vis)
    cu = np.arange(5, 60, 2)
    cv = (cu * 7) % 64
    assert np.array_equal(o.grid_cells(g, ks, b, vis, cu, cv), G[cv, cu])


# --------------------------------------------------------------- forward model (prediction)
def test_image_to_grid_is_the_adjoint_of_the_dirty_image():
    """For any complex grid G and real image Y: <dirty_image(G), Y> = Re <G, image_to_grid(Y)>
    (same taper, disc and weight sum).  A wrong sign of the exponent, a missing shift, a
    taper multiplied instead of divided, or a different disc breaks the identity."""
    N = 48
    g = o.Geometry(N, np.deg2rad(3.0) / N, 4, 7, 1, 0.0, 256)
    rng = np.random.default_rng(21)
    tap = o.gaussian_taper(g, 0.25)
    G = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    Y = rng.normal(size=(N, N))
    ws = 3.7
    lhs = float(np.sum(o.dirty_image(g, G, tap, ws) * Y))
    rhs = float(np.real(np.vdot(o.image_to_grid(g, Y, tap, ws), G)))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # and the identity is not vacuous: the transposed (unshifted) grid fails it
    bad = float(np.real(np.vdot(o.image_to_grid(g, Y.T, tap, ws), G)))
    assert abs(bad - lhs) > 1e-3 * abs(lhs)


def _prediction_error(os_, planes_count, seed=5, S_max=15, on_grid=False):
    """Max error of the w-projection prediction (degridding of the tapered, transformed model
    image) against the non-coplanar visibility equation (Eq. 2) summed directly over point
    sources placed on pixel centres, relative to the largest visibility; with the bound the
    oversampling quantisation alone allows.  on_grid: (u, v) on the fine grid (multiples of
    du/os) and w on the plane values, so that neither offset is quantised."""
    N = 64
    dl = np.deg2rad(4.0) / N
    g = o.Geometry(N, dl, os_, S_max, 2, 0.001, 512)
    rng = np.random.default_rng(seed)
    V = 600
    rad = (N / 2 - S_max - 2) * g.du * np.sqrt(rng.random(V))
    th = 2 * np.pi * rng.random(V)
    u, v = rad * np.cos(th), rad * np.sin(th)
    planes = np.linspace(0, 400, planes_count) if planes_count > 1 else np.array([0.0])
    w = rng.uniform(-400, 400, V)
    if on_grid:
        u = np.rint(u * os_ / g.du) * g.du / os_
        v = np.rint(v * os_ / g.du) * g.du / os_
        w = planes[rng.integers(0, len(planes), V)] * rng.choice([-1.0, 1.0], V)
    uvw = np.stack([u, v, w], 1).astype(np.float32)
    pix = [(N // 2 + 9, N // 2 - 5, 1.0), (N // 2 - 12, N // 2 + 7, 0.6), (N // 2 + 3, N // 2 + 14, 0.8)]
    img = np.zeros((N, N))
    for il, im, f in pix:
        img[im, il] = f
    tap = o.gaussian_taper(g, 0.2)
    pred = o.predict_vis(g, img, tap, planes, None, uvw)
    u, v, w = (uvw[:, k].astype(np.float64) for k in range(3))
    direct = np.zeros(V, dtype=np.complex128)
    bound = 0.0
    for il, im, f in pix:
        l, m = (il - N // 2) * dl, (im - N // 2) * dl
        n = np.sqrt(1.0 - l * l - m * m)
        direct += f * np.exp(-2j * np.pi * (u * l + v * m + w * (n - 1.0)))
        # |du|, |dv| <= du / (2 os): phase error <= pi (|il - N/2| + |im - N/2|) / (N os)
        bound += f * np.pi * (abs(il - N // 2) + abs(im - N // 2)) / (N * os_)
    scale = np.abs(direct).max()
    return np.abs(pred - direct).max() / scale, bound / scale


def test_prediction_matches_direct_visibility_equation():
    """Eq. 2 evaluated directly vs the oracle's w-projection prediction.  Off the fine grid the
    gap is dominated by the oversampling quantisation of each visibility's offset: it stays
    under that term's bound, halves when os doubles and grows without w-correction.  With
    (u, v) on the fine grid and w on the planes nothing is quantised, and what remains (kernel
    truncation at 0.1 %, spline interpolation, aliasing of the taper) is far smaller."""
    e8, b8 = _prediction_error(8, 17)
    assert e8 < b8
    e16, _ = _prediction_error(16, 17)
    assert 0.35 * e8 < e16 < 0.65 * e8
    e2, _ = _prediction_error(2, 17)
    assert e2 > 3 * e8
    e_off, _ = _prediction_error(8, 1)
    assert e_off > 3 * e8
    exact8, _ = _prediction_error(8, 17, on_grid=True)
    assert exact8 < 5e-3 and exact8 < 0.1 * e8
