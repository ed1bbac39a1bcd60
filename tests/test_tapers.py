"""Anti-aliasing functions: the radially symmetric prolate spheroidal taper (the alternative
the paper names beside its Gaussian, Section 5: radial symmetry enforced by taking the 1D
function along the radius), pinned as a finite-Fourier-transform eigenfunction, and its
aliasing compared with a Gaussian of the same kernel support on the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import oracle as o

sp = pytest.importorskip("scipy.special")


def test_pswf_is_a_finite_fourier_eigenfunction():
    """psi(c, x) satisfies int_{-1}^{1} exp(j c x t) psi(t) dt = lambda psi(x): the ratio is
    the same at every x (Gauss-Legendre quadrature, psi even in t); the taper samples are
    psi at x = r_i / r_max."""
    c = 3.0 * np.pi
    t, wq = np.polynomial.legendre.leggauss(200)
    psi_t = sp.pro_ang1(0, 0, c, np.abs(t))[0]
    ratios = []
    for x in (0.0, 0.2, 0.45, 0.7, 0.9):
        lhs = np.sum(wq * np.exp(1j * c * x * t) * psi_t)
        ratios.append(lhs / sp.pro_ang1(0, 0, c, x)[0])
    ratios = np.array(ratios)
    assert np.abs(ratios.imag).max() < 1e-10 * np.abs(ratios).max()
    assert np.ptp(ratios.real) < 1e-8 * np.abs(ratios.real).max()
    N, dl, R = 64, np.deg2rad(4.0) / 64, 512
    tap = synth.pswf_taper_samples(N, dl, R, c)
    x = (np.arange(R) + 0.5) / R
    assert np.allclose(tap, sp.pro_ang1(0, 0, c, x)[0], rtol=1e-12, atol=0)


def _alias_error(tap_fn, l0_frac):
    """Max error, over the inner 3/4 of the circle, of the w-projection dirty image of one
    unit source outside the field (at l = l0_frac FOV, aliasing into the image) against the
    brute-force direct image; w = 0, so only the anti-aliasing function matters."""
    N, S_max = 64, 7
    g = o.Geometry(N, np.deg2rad(4.0) / N, 8, S_max, 1, 0.01, 512)
    tap = tap_fn(g)
    rng = np.random.default_rng(3)
    V = 3000
    rad = (N / 2 - S_max - 2) * g.du * np.sqrt(rng.random(V))
    th = 2 * np.pi * rng.random(V)
    uvw = np.stack([rad * np.cos(th), rad * np.sin(th), np.zeros(V)], 1).astype(np.float32)
    vis = np.exp(-2j * np.pi * uvw[:, 0].astype(np.float64) * l0_frac * g.fov).astype(np.complex64)
    planes = np.array([0.0])
    ks = o.wkernels(g, tap, planes)
    b = o.bin_vis(g, uvw, planes, ks.support)
    img = o.dirty_image(g, o.grid(g, ks, b, vis), tap, float((b.drop == 0).sum()))
    im_, il_ = np.nonzero(o.disc_mask(g))
    inner = np.hypot(il_ - N / 2, im_ - N / 2) < 0.75 * N / 2
    im_, il_ = im_[inner], il_[inner]
    ref = o.dft_image(g, uvw, vis, pixels=(il_, im_))
    return np.abs(img[im_, il_] - ref).max(), int(ks.support[0])


@pytest.mark.parametrize("l0_frac", [0.7, 0.9])
def test_pswf_taper_aliases_less_than_gaussian_of_equal_support(l0_frac):
    """At the same 1 % kernel support (3 cells) the prolate taper leaves about half the alias
    error of a Gaussian (sigma = FOV / 2 pi, uv sigma one cell)."""
    N, dl = 64, np.deg2rad(4.0) / 64
    e_p, s_p = _alias_error(lambda g: synth.pswf_taper_samples(N, dl, 512), l0_frac)
    e_g, s_g = _alias_error(lambda g: o.gaussian_taper(g, 1.0 / (2.0 * np.pi)), l0_frac)
    assert s_p == s_g == 3
    assert e_p < 0.85 * e_g
