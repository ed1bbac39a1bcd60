"""FP64 CPU oracle for Hankel-accelerated w-projection (Lucas, Skipper & Scaife 2019).

TEST INFRASTRUCTURE ONLY.  This module and the C file beside it are the plain, slow,
obviously-correct reference that the CUDA library is checked against.  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It imports nothing from the CUDA package and the CUDA package never
imports it; the two share only the seeded input generators of ``synth``.

Everything is double precision.  The loops live in ``wproj_oracle.c`` (compiled on
first use with gcc, no fast-math, no FP contraction); the two FFT steps (the 2D-FFT
kernel generator of Alg. 1 and the inverse transform of the dirty image) use
``numpy.fft`` as a library primitive.

Notation (Sections 3-4 of the paper):
    N      image side (pixels), dl cell size (direction cosine), FOV = N*dl
    du     uv cell = 1/FOV (wavelengths)
    r_max  radius of the circular image region = FOV/2 (Section 6: the valid region of
           the Hankel dirty image is the circle whose diameter is the image size)
    R      radial samples of the image-domain functions, r_i = (i+1/2) r_max/R
    os     oversampling; the radial kernel line is sampled at rho_k = k du/os
    K_out  radial kernel samples = os*(S_max+2) rounded up to a multiple of 128
    S      kernel support (half-width in cells), full width 2S+1 (Section 5)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wproj_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (plain gcc, FP64, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            D = ctypes.c_double
            I = ctypes.c_int
            L = ctypes.c_int64
            P = ctypes.c_void_p
            lib.or_j0.restype = D
            lib.or_j0.argtypes = [D]
            lib.or_j0_array.argtypes = [L, P, P]
            lib.or_hankel_matrix.argtypes = [I, D, I, P, P]
            lib.or_hankel_apply.argtypes = [I, I, P, P, P]
            lib.or_hankel_direct.argtypes = [I, D, P, I, P, P]
            lib.or_screen.argtypes = [I, D, P, D, P]
            lib.or_support.restype = I
            lib.or_support.argtypes = [I, P, D, I, I, I]
            lib.or_spline_m.argtypes = [I, P, D, P]
            lib.or_spline_eval_array.argtypes = [I, P, P, D, I, L, P, P]
            lib.or_resample.argtypes = [I, P, P, I, I, I, P]
            lib.or_bin.argtypes = [L, P, I, P, P, I, D, I, P, P, P, P, P, P, P]
            lib.or_grid.argtypes = [L, P, P, P, P, P, P, P, P, P, P, P, P, I, I, P]
            lib.or_degrid.argtypes = [L, P, P, P, P, P, P, P, P, P, P, I, I, P, P]
            lib.or_dft_image.argtypes = [L, P, P, P, I, D, I, P, P, P]
            lib.or_grid_cells.argtypes = [L, P, P, P, P, P, P, P, P, P, P, I, P, P, I, I, I, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------------------
# Geometry
# --------------------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Geometry:
    """Imager settings of Section 5 (image size, cell size, oversampling, support)."""

    image_size: int          # N
    cell_size: float         # dl, direction cosine per pixel
    oversampling: int = 8    # os
    max_support: int = 15    # S_max (half-width)
    min_support: int = 3     # S_min
    trunc_frac: float = 0.01 # tau (Section 3.1: 1 %)
    radial_samples: int = 512  # R
    interp: int = 0          # 0 cubic spline, 1 linear (Section 4.3.2)

    @property
    def fov(self) -> float:
        return self.image_size * self.cell_size

    @property
    def du(self) -> float:
        return 1.0 / (self.image_size * self.cell_size)

    @property
    def r_max(self) -> float:
        return 0.5 * self.image_size * self.cell_size

    @property
    def k_out(self) -> int:
        k = self.oversampling * (self.max_support + 2)
        return ((k + 127) // 128) * 128

    def rho(self) -> np.ndarray:
        """Radial kernel sample positions rho_k = k du / os (wavelengths)."""
        return np.arange(self.k_out, dtype=np.float64) * (self.du / self.oversampling)

    def r_nodes(self) -> np.ndarray:
        R = self.radial_samples
        return (np.arange(R, dtype=np.float64) + 0.5) * (self.r_max / R)


def gaussian_taper(geom: Geometry, sigma_frac: float = 0.3) -> np.ndarray:
    """Gaussian anti-aliasing function (Section 5) sampled at the radial nodes r_i.

    Reading: the paper does not give the width; sigma = 0.3 FOV by default."""
    r = geom.r_nodes()
    s = sigma_frac * geom.fov
    return np.exp(-0.5 * (r / s) ** 2)


def taper_at(geom: Geometry, taper: np.ndarray, r: np.ndarray) -> np.ndarray:
    """t(r) between the nodes: linear interpolation of the sampled taper, clamped at the
    end nodes, zero beyond r_max (the disc the Hankel transform integrates over)."""
    R = geom.radial_samples
    x = np.asarray(r, dtype=np.float64) / (geom.r_max / R) - 0.5
    x = np.clip(x, 0.0, R - 1.0)
    i0 = np.minimum(np.floor(x).astype(np.int64), R - 2)
    a = x - i0
    t = (1.0 - a) * taper[i0] + a * taper[i0 + 1]
    return np.where(np.asarray(r) <= geom.r_max, t, 0.0)


def workspace_size(max_support: int) -> int:
    """Workspace undersampling (Section 4.2): power of two >= the full kernel width 2S+1."""
    full = 2 * max_support + 1
    m = 1
    while m < full:
        m *= 2
    return m


# --------------------------------------------------------------------------------------
# Bessel J0 and the Hankel transform
# --------------------------------------------------------------------------------------
def j0(x) -> np.ndarray:
    x = _f64(np.atleast_1d(x))
    out = np.empty_like(x)
    _load().or_j0_array(x.size, _p(x), _p(out))
    return out


_H_CACHE: dict = {}


def hankel_matrix(R: int, r_max: float, rho: np.ndarray) -> np.ndarray:
    """H[k][i] = 2 pi r_i dr J0(2 pi rho_k r_i) (Section 4.3, matrix form)."""
    rho = _f64(rho)
    key = (R, float(r_max), rho.size, rho.tobytes()[:64], float(rho[-1]) if rho.size else 0.0)
    H = _H_CACHE.get(key)
    if H is None:
        H = np.empty((rho.size, R), dtype=np.float64)
        _load().or_hankel_matrix(R, float(r_max), rho.size, _p(rho), _p(H))
        if len(_H_CACHE) > 4:
            _H_CACHE.clear()
        _H_CACHE[key] = H
    return H


def hankel(f: np.ndarray, r_max: float, rho: np.ndarray) -> np.ndarray:
    """Order-0 Hankel transform (2 pi normalised) of samples f(r_i) at radii rho."""
    f = _c128(f)
    rho = _f64(rho)
    out = np.empty(rho.size, dtype=np.complex128)
    _load().or_hankel_direct(f.size, float(r_max), _p(f.view(np.float64)), rho.size, _p(rho),
                             _p(out.view(np.float64)))
    return out


def hankel_apply(H: np.ndarray, f: np.ndarray) -> np.ndarray:
    f = _c128(f)
    H = _f64(H)
    out = np.empty(H.shape[0], dtype=np.complex128)
    _load().or_hankel_apply(H.shape[1], H.shape[0], _p(H), _p(f.view(np.float64)),
                            _p(out.view(np.float64)))
    return out


def screen(geom: Geometry, taper: np.ndarray, w: float) -> np.ndarray:
    """Image-domain convolution function on the radial line: taper x w-screen (Alg. 2)."""
    taper = _f64(taper)
    f = np.empty(geom.radial_samples, dtype=np.complex128)
    _load().or_screen(geom.radial_samples, geom.r_max, _p(taper), float(w), _p(f.view(np.float64)))
    return f


def radial_kernel(geom: Geometry, taper: np.ndarray, w: float) -> np.ndarray:
    """Radial gridding-kernel line C_w(rho_k), k < K_out, in tap units (times du^2, so that
    each 2D kernel sums to about t(0) = 1).  Hankel transform replaces the 2D FFT (Alg. 2)."""
    H = hankel_matrix(geom.radial_samples, geom.r_max, geom.rho())
    return hankel_apply(H, screen(geom, taper, w)) * geom.du ** 2


def support(geom: Geometry, C: np.ndarray) -> int:
    C = _c128(C)
    return int(_load().or_support(C.size, _p(C.view(np.float64)), float(geom.trunc_frac),
                                  geom.oversampling, geom.min_support, geom.max_support))


def spline_m(y: np.ndarray) -> np.ndarray:
    """Cubic-spline second derivatives on unit node spacing (Section 4.3.2)."""
    y = _c128(y)
    m = np.empty_like(y)
    _load().or_spline_m(y.size, _p(y.view(np.float64)), 1.0, _p(m.view(np.float64)))
    return m


def spline_eval(y: np.ndarray, m: np.ndarray, x: np.ndarray, interp: int = 0) -> np.ndarray:
    y = _c128(y)
    m = _c128(m)
    x = _f64(x)
    out = np.empty(x.size, dtype=np.complex128)
    _load().or_spline_eval_array(y.size, _p(y.view(np.float64)), _p(m.view(np.float64)), 1.0,
                                 int(interp), x.size, _p(x), _p(out.view(np.float64)))
    return out


def resample(geom: Geometry, C: np.ndarray, S: int) -> np.ndarray:
    """Oversampled kernel cache of one plane, shape [os][os][2S+1][2S+1] complex128."""
    C = _c128(C)
    m = spline_m(C) if geom.interp == 0 else np.zeros_like(C)
    os_ = geom.oversampling
    W = 2 * S + 1
    out = np.empty((os_, os_, W, W), dtype=np.complex128)
    _load().or_resample(C.size, _p(C.view(np.float64)), _p(m.view(np.float64)), os_, int(S),
                        int(geom.interp), _p(out.view(np.float64)))
    return out


@dataclasses.dataclass
class KernelSet:
    """Oversampled kernel caches of all |w|-planes (Alg. 2 kernel cache)."""

    w_planes: np.ndarray     # |w| plane values, ascending
    radial: np.ndarray       # [P][K_out] complex128
    support: np.ndarray      # [P] int32
    offsets: np.ndarray      # [P+1] int64, start of each plane (complex elements)
    cache: np.ndarray        # flat complex128


def layout(geom: Geometry, support_arr) -> np.ndarray:
    os2 = geom.oversampling ** 2
    sizes = [os2 * (2 * int(s) + 1) ** 2 for s in support_arr]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def wkernels(geom: Geometry, taper: np.ndarray, w_planes, supports=None, with_cache: bool = True,
             route: str = "hankel") -> KernelSet:
    """w-kernels for every plane: radial line, truncate, spline, resample.  The radial line
    comes from the matrix Hankel transform (route="hankel", Section 4.3) or from the
    projection-slice theorem on the undersampled workspace (route="projslice", Section 4.3.1).
    with_cache=False stops after the radial lines and supports (cache left empty)."""
    w_planes = _f64(w_planes)
    line = radial_kernel if route == "hankel" else projslice_radial
    radial = np.stack([line(geom, taper, w) for w in w_planes])
    if supports is None:
        sup = np.array([support(geom, radial[p]) for p in range(len(w_planes))], dtype=np.int32)
    else:
        sup = np.asarray(supports, dtype=np.int32)
    off = layout(geom, sup)
    if not with_cache:
        return KernelSet(w_planes, radial, sup, off, np.empty(0, dtype=np.complex128))
    cache = np.empty(int(off[-1]), dtype=np.complex128)
    for p in range(len(w_planes)):
        cache[off[p]:off[p + 1]] = resample(geom, radial[p], int(sup[p])).ravel()
    return KernelSet(w_planes, radial, sup, off, cache)


# --------------------------------------------------------------------------------------
# Standard w-projection kernels by 2D FFT (Alg. 1 steps 4-11, workspace undersampling)
# --------------------------------------------------------------------------------------
def workspace_image(geom: Geometry, taper: np.ndarray, w: float):
    """Image-domain convolution function on the undersampled M x M workspace (Section 4.2;
    Alg. 1 steps 5-8, Alg. 2 steps 4-8): taper x w-screen at the pixel centres l = j FOV/M,
    j = -M/2 .. M/2-1, zero outside the disc r <= r_max = (M/2) FOV/M (decided on the integer
    offsets).  Returns (f [m][l], j, pixel size)."""
    M = workspace_size(geom.max_support)
    dlw = geom.fov / M
    j = np.arange(M) - M // 2
    l = j * dlw
    L, Mm = np.meshgrid(l, l, indexing="xy")      # [m][l]
    r = np.hypot(L, Mm)
    inside = (j[None, :] ** 2 + j[:, None] ** 2) <= (M // 2) ** 2
    t = np.where(inside, taper_at(geom, taper, np.minimum(r, geom.r_max)), 0.0)
    n = np.sqrt(1.0 - r * r)
    return t * np.exp(2j * np.pi * w * (n - 1.0)), j, dlw


def projslice_radial(geom: Geometry, taper: np.ndarray, w: float) -> np.ndarray:
    """Radial kernel line by the projection-slice theorem (Section 4.3.1, Alg. 2 steps 9-12):
    the workspace image is projected onto the l axis (summed over m), zero padded to M*os and
    transformed by a 1D FFT; sample k sits at uv offset k du/os on the v = 0 slice.  Scaled
    like the 2D route: (FOV/M)^2 du^2.  Samples k >= M*os wrap periodically."""
    f, j, dlw = workspace_image(geom, taper, w)
    Lp = f.shape[0] * geom.oversampling
    X = np.zeros(Lp, dtype=np.complex128)
    X[j % Lp] = f.sum(axis=0)
    Y = np.fft.fft(X) * (dlw ** 2) * geom.du ** 2
    return Y[np.arange(geom.k_out) % Lp]


def fft_wkernel(geom: Geometry, taper: np.ndarray, w: float, S: int, circular: bool = True) -> np.ndarray:
    """Kernel cache of one plane by the 2D FFT route (Alg. 1 with Section 4.2).

    The M x M workspace (M = power of two >= 2 S_max + 1) samples the image-domain
    product taper x screen over the whole FOV (pixel FOV/M), is zero padded to M*os,
    and transformed; sample a of the result sits at uv offset a du/os.  Sub-kernel
    (fu, fv), tap (jx, jy) is the sample at offset (os (jx-S) - fu, os (jy-S) - fv).
    The image-domain function is zero outside the disc r <= r_max so that the two
    routes transform the same function; with circular=True taps beyond radius S are
    zeroed as in the Hankel route."""
    f, j, dlw = workspace_image(geom, taper, w)
    M = f.shape[0]
    os_ = geom.oversampling
    Lp = M * os_
    X = np.zeros((Lp, Lp), dtype=np.complex128)
    X[np.ix_(j % Lp, j % Lp)] = f
    Y = np.fft.fft2(X) * (dlw ** 2) * geom.du ** 2
    W = 2 * S + 1
    jj = np.arange(W) - S
    out = np.empty((os_, os_, W, W), dtype=np.complex128)
    for fv in range(os_):
        ay = (os_ * jj - fv) % Lp
        for fu in range(os_):
            ax = (os_ * jj - fu) % Lp
            out[fv, fu] = Y[np.ix_(ay, ax)]
    if circular:
        fvv, fuu, jy, jx = np.meshgrid(np.arange(os_), np.arange(os_), jj, jj, indexing="ij")
        q = (os_ * jx - fuu) ** 2 + (os_ * jy - fvv) ** 2
        out[q > (os_ * S) ** 2] = 0.0
    return out


# --------------------------------------------------------------------------------------
# Binning, gridding, degridding, dirty image
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Bins:
    plane: np.ndarray
    conj: np.ndarray
    iu: np.ndarray
    iv: np.ndarray
    fu: np.ndarray
    fv: np.ndarray
    drop: np.ndarray


def bin_vis(geom: Geometry, uvw: np.ndarray, w_planes, supports) -> Bins:
    uvw = np.ascontiguousarray(uvw, dtype=np.float32).reshape(-1, 3)
    V = uvw.shape[0]
    wp = _f64(w_planes)
    sup = np.ascontiguousarray(supports, dtype=np.int32)
    arr = [np.zeros(V, dtype=np.int32) for _ in range(7)]
    _load().or_bin(V, _p(uvw), wp.size, _p(wp), _p(sup), geom.image_size, geom.du,
                   geom.oversampling, *[_p(a) for a in arr])
    return Bins(*arr)


def grid(geom: Geometry, ks: KernelSet, bins: Bins, vis: np.ndarray, wt=None) -> np.ndarray:
    """uv-grid [N][N] complex128 (rows v, columns u) of the gridded visibilities."""
    N = geom.image_size
    vis = np.ascontiguousarray(vis, dtype=np.complex64).view(np.float32)
    wtp = None
    if wt is not None:
        wt = np.ascontiguousarray(wt, dtype=np.float32)
        wtp = _p(wt)
    g = np.zeros((N, N), dtype=np.complex128)
    cache = _c128(ks.cache)
    off = np.ascontiguousarray(ks.offsets, dtype=np.int64)
    sup = np.ascontiguousarray(ks.support, dtype=np.int32)
    _load().or_grid(bins.plane.size, _p(bins.plane), _p(bins.conj), _p(bins.iu), _p(bins.iv),
                    _p(bins.fu), _p(bins.fv), _p(bins.drop), _p(vis), wtp, _p(sup), _p(off),
                    _p(cache.view(np.float64)), geom.oversampling, N, _p(g.view(np.float64)))
    return g


def degrid(geom: Geometry, ks: KernelSet, bins: Bins, g: np.ndarray) -> np.ndarray:
    N = geom.image_size
    g = _c128(g)
    out = np.empty(bins.plane.size, dtype=np.complex128)
    cache = _c128(ks.cache)
    off = np.ascontiguousarray(ks.offsets, dtype=np.int64)
    sup = np.ascontiguousarray(ks.support, dtype=np.int32)
    _load().or_degrid(bins.plane.size, _p(bins.plane), _p(bins.conj), _p(bins.iu), _p(bins.iv),
                      _p(bins.fu), _p(bins.fv), _p(bins.drop), _p(sup), _p(off),
                      _p(cache.view(np.float64)), geom.oversampling, N, _p(g.view(np.float64)),
                      _p(out.view(np.float64)))
    return out


def disc_mask(geom: Geometry) -> np.ndarray:
    """Pixels inside the circular region (diameter = image size): integer test
    (il - N/2)^2 + (im - N/2)^2 <= (N/2)^2."""
    N = geom.image_size
    d = np.arange(N) - N // 2
    return (d[None, :] ** 2 + d[:, None] ** 2) <= (N // 2) ** 2


def pixel_radius(geom: Geometry) -> np.ndarray:
    N = geom.image_size
    d = (np.arange(N) - N // 2).astype(np.float64)
    return geom.cell_size * np.sqrt(d[None, :] ** 2 + d[:, None] ** 2)


def dirty_image(geom: Geometry, g: np.ndarray, taper: np.ndarray, weight_sum: float) -> np.ndarray:
    """Dirty image [N][N] (rows m, columns l): inverse transform of the grid, divided by the
    anti-aliasing function and the weight sum (Section 3), zero outside the disc.

    I(l, m) = Re sum_{u,v} grid(u, v) exp(+2 pi j (u l + v m)) / (t(r) sum wt)."""
    N = geom.image_size
    img = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g))) * (N * N)
    t = taper_at(geom, taper, pixel_radius(geom))
    inside = disc_mask(geom)
    out = np.zeros((N, N), dtype=np.float64)
    out[inside] = img.real[inside] / (t[inside] * weight_sum)
    return out


def dft_image(geom: Geometry, uvw: np.ndarray, vis: np.ndarray, wt=None, pixels=None) -> np.ndarray:
    """Brute-force image: adjoint of Eq. 2 evaluated pixel by pixel.  pixels: (il, im) int
    arrays; default all pixels inside the disc.  Returns the values at those pixels."""
    N = geom.image_size
    uvw = np.ascontiguousarray(uvw, dtype=np.float32).reshape(-1, 3)
    vis = np.ascontiguousarray(vis, dtype=np.complex64).view(np.float32)
    wtp = None
    if wt is not None:
        wt = np.ascontiguousarray(wt, dtype=np.float32)
        wtp = _p(wt)
    if pixels is None:
        im_, il_ = np.nonzero(disc_mask(geom))
    else:
        il_, im_ = pixels
    il_ = np.ascontiguousarray(il_, dtype=np.int32)
    im_ = np.ascontiguousarray(im_, dtype=np.int32)
    out = np.empty(il_.size, dtype=np.float64)
    _load().or_dft_image(uvw.shape[0], _p(uvw), _p(vis), wtp, N, geom.cell_size, il_.size,
                         _p(il_), _p(im_), _p(out))
    return out


def mean_w_planes(w: np.ndarray, P: int) -> np.ndarray:
    """Plane values as in Alg. 2 steps 1-3: sort |w|, cut into P equal-count chunks, take
    each chunk's mean (the paper's default, `wplanes_median: false`, Section 5).  Reading:
    non-finite |w| take no part (they are dropped at binning); a chunk left empty (fewer
    finite values than planes) takes the largest finite |w| (0 if none), so the values stay
    ascending."""
    aw = np.sort(np.abs(np.asarray(w, dtype=np.float64)))
    aw = aw[np.isfinite(aw)]
    top = aw[-1] if aw.size else 0.0
    chunks = np.array_split(aw, P)
    return np.array([c.mean() if c.size else top for c in chunks], dtype=np.float64)


# --------------------------------------------------------------------------------------
# Visibility prediction from a model image (the forward model whose gradients the CUDA
# path differentiates): the adjoint pair of the dirty image and of gridding.
# --------------------------------------------------------------------------------------
def image_to_grid(geom: Geometry, image: np.ndarray, taper: np.ndarray, weight_sum: float = 1.0) -> np.ndarray:
    """grid[v][u] = sum over pixels inside the circle of I / (t(r) wsum)
    exp(-2 pi j ((u - N/2)(l - N/2) + (v - N/2)(m - N/2)) / N): the adjoint of the linear part
    of dirty_image (Section 3)."""
    t = taper_at(geom, taper, pixel_radius(geom))
    inside = disc_mask(geom)
    X = np.zeros_like(np.asarray(image, dtype=np.float64))
    X[inside] = np.asarray(image, dtype=np.float64)[inside] / (t[inside] * weight_sum)
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(X)))


def predict_vis(geom: Geometry, image: np.ndarray, taper: np.ndarray, w_planes, supports, uvw: np.ndarray,
                weight_sum: float = 1.0) -> np.ndarray:
    """V = degrid(kernels(taper), image_to_grid(image; taper)), all in FP64."""
    ks = wkernels(geom, taper, w_planes, supports=supports)
    b = bin_vis(geom, uvw, w_planes, ks.support)
    return degrid(geom, ks, b, image_to_grid(geom, image, taper, weight_sum))


def grid_cells(geom: Geometry, ks: KernelSet, bins: Bins, vis: np.ndarray, cells_u, cells_v, wt=None) -> np.ndarray:
    """Gridded values at the listed cells, taps evaluated from the radial lines directly."""
    vis = np.ascontiguousarray(vis, dtype=np.complex64).view(np.float32)
    wtp = None
    if wt is not None:
        wt = np.ascontiguousarray(wt, dtype=np.float32)
        wtp = _p(wt)
    radial = _c128(ks.radial)
    m = np.stack([spline_m(r) for r in radial]) if geom.interp == 0 else np.zeros_like(radial)
    m = _c128(m)
    cu = np.ascontiguousarray(cells_u, dtype=np.int32)
    cv = np.ascontiguousarray(cells_v, dtype=np.int32)
    sup = np.ascontiguousarray(ks.support, dtype=np.int32)
    out = np.empty(cu.size, dtype=np.complex128)
    _load().or_grid_cells(bins.plane.size, _p(bins.plane), _p(bins.conj), _p(bins.iu), _p(bins.iv), _p(bins.fu),
                          _p(bins.fv), _p(bins.drop), _p(vis), wtp, _p(sup), radial.shape[1],
                          _p(radial.view(np.float64)), _p(m.view(np.float64)), int(geom.interp), geom.oversampling,
                          cu.size, _p(cu), _p(cv), _p(out.view(np.float64)))
    return out
