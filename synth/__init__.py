"""Seeded synthetic inputs shaped like the paper's imaging workloads.

This module only makes inputs: visibility coordinates (uvw), point-source sky models
and the visibilities they produce through the measurement equation (Eq. 2), plus the
radial anti-aliasing taper samples.  It contains none of the w-projection method
(no kernels, no Hankel transform, no gridding) and is shared by the CPU oracle, the
tests and the benchmark so that both sides see identical inputs.

Every generator takes an explicit integer seed (numpy PCG64).  Arrays are numpy,
float32 for uvw (wavelengths, [V][3]) and complex64 for visibilities, as the CUDA
path consumes them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299792458.0


@dataclasses.dataclass
class Sky:
    l: np.ndarray      # direction cosines
    m: np.ndarray
    flux: np.ndarray   # Jy (apparent)


def gaussian_taper_samples(image_size: int, cell_size: float, radial_samples: int,
                           sigma_frac: float = 0.3) -> np.ndarray:
    """Gaussian anti-aliasing function t(r) = exp(-r^2 / (2 sigma^2)), sigma = sigma_frac * FOV,
    sampled at the radial nodes r_i = (i + 1/2) r_max / R, r_max = FOV / 2 (float64)."""
    fov = image_size * cell_size
    r_max = 0.5 * fov
    r = (np.arange(radial_samples, dtype=np.float64) + 0.5) * (r_max / radial_samples)
    s = sigma_frac * fov
    return np.exp(-0.5 * (r / s) ** 2)


def pswf_taper_samples(image_size: int, cell_size: float, radial_samples: int,
                       c: float = 3.0 * np.pi) -> np.ndarray:
    """Radially symmetric prolate spheroidal anti-aliasing function: the order-0 angular
    prolate spheroidal function psi(c, x) (scipy's pro_ang1, normalised to psi(0) = 1) taken
    along the radius, x = r / r_max, sampled at the radial nodes r_i = (i + 1/2) r_max / R.
    Its transform is concentrated within about c / pi uv cells; c = 3 pi matches the
    classic six-cell-wide gridding function."""
    import scipy.special as sp

    x = (np.arange(radial_samples, dtype=np.float64) + 0.5) / radial_samples
    psi = sp.pro_ang1(0, 0, c, x)[0]
    return psi / sp.pro_ang1(0, 0, c, 0.0)[0]


def uniform_disc_uvw(V: int, uv_radius: float, w_max: float, seed: int) -> np.ndarray:
    """(u, v) uniform in a disc of radius uv_radius, w uniform in [-w_max, w_max]."""
    rng = np.random.default_rng(seed)
    rad = uv_radius * np.sqrt(rng.random(V))
    th = 2.0 * np.pi * rng.random(V)
    w = rng.uniform(-w_max, w_max, V)
    return np.stack([rad * np.cos(th), rad * np.sin(th), w], axis=1).astype(np.float32)


def sources_in_disc(n: int, radius: float, seed: int, flux_lo: float = 0.1, flux_hi: float = 1.0,
                    log_uniform: bool = False) -> Sky:
    """n point sources uniform in the disc of the given radius (direction cosines)."""
    rng = np.random.default_rng(seed)
    rad = radius * np.sqrt(rng.random(n))
    th = 2.0 * np.pi * rng.random(n)
    if log_uniform:
        flux = np.exp(rng.uniform(np.log(flux_lo), np.log(flux_hi), n))
    else:
        flux = rng.uniform(flux_lo, flux_hi, n)
    return Sky(rad * np.cos(th), rad * np.sin(th), flux)


def predict(uvw: np.ndarray, sky: Sky, chunk: int = 1 << 16) -> np.ndarray:
    """Visibilities of point sources by direct evaluation of the non-coplanar measurement
    equation (Eq. 2): V = sum_s F_s exp(-2 pi j (u l_s + v m_s + w (n_s - 1))), FP64.
    The 1/n factor is absorbed in the apparent flux F_s."""
    uvw64 = np.asarray(uvw, dtype=np.float64).reshape(-1, 3)
    n = np.sqrt(1.0 - sky.l ** 2 - sky.m ** 2)
    out = np.empty(uvw64.shape[0], dtype=np.complex128)
    for a in range(0, uvw64.shape[0], chunk):
        u = uvw64[a:a + chunk, 0:1]
        v = uvw64[a:a + chunk, 1:2]
        w = uvw64[a:a + chunk, 2:3]
        ph = -2.0 * np.pi * (u * sky.l[None] + v * sky.m[None] + w * (n[None] - 1.0))
        out[a:a + chunk] = (sky.flux[None] * np.exp(1j * ph)).sum(axis=1)
    return out.astype(np.complex64)


def predict_torch(uvw, sky: Sky, device, chunk: int = 1 << 18):
    """Same as predict() with torch FP64 on `device` (for the multi-million visibility
    workload); returns a complex64 torch tensor on that device."""
    import torch

    uvw64 = torch.as_tensor(np.asarray(uvw), device=device).to(torch.float64).reshape(-1, 3)
    l = torch.as_tensor(sky.l, device=device, dtype=torch.float64)
    m = torch.as_tensor(sky.m, device=device, dtype=torch.float64)
    f = torch.as_tensor(sky.flux, device=device, dtype=torch.float64)
    n = torch.sqrt(1.0 - l * l - m * m)
    out = torch.empty(uvw64.shape[0], dtype=torch.complex64, device=device)
    for a in range(0, uvw64.shape[0], chunk):
        u = uvw64[a:a + chunk, 0:1]
        v = uvw64[a:a + chunk, 1:2]
        w = uvw64[a:a + chunk, 2:3]
        ph = -2.0 * math.pi * (u * l[None] + v * m[None] + w * (n[None] - 1.0))
        re = (f[None] * torch.cos(ph)).sum(dim=1)
        im = (f[None] * torch.sin(ph)).sum(dim=1)
        out[a:a + chunk] = torch.complex(re, im).to(torch.complex64)
    return out


def add_noise(vis: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    nz = rng.normal(0.0, sigma, (vis.shape[0], 2))
    return (vis + (nz[:, 0] + 1j * nz[:, 1])).astype(np.complex64)


def array_layout(n_ant: int, radius_m: float, seed: int) -> np.ndarray:
    """Antenna (east, north) positions uniform in a disc of radius radius_m, flat array."""
    rng = np.random.default_rng(seed)
    rad = radius_m * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    return np.stack([rad * np.cos(th), rad * np.sin(th), np.zeros(n_ant)], axis=1)


def track_uvw(n_ant: int = 64, radius_m: float = 5000.0, lat_deg: float = -30.0,
              dec_deg: float = -30.0, hours: float = 8.0, n_dumps: int = 4162,
              freq_hz: float = 1.4e9, seed: int = 3, max_vis: int | None = None) -> np.ndarray:
    """Earth-rotation tracks of every baseline (baseline-major, time-ordered), in wavelengths.

    Local (east, north, up) baselines are rotated to equatorial (X, Y, Z) for latitude lat,
    then to (u, v, w) for hour angle H and declination dec (standard interferometry
    geometry).  Hour angles span [-hours/2, +hours/2]."""
    enu = array_layout(n_ant, radius_m, seed)
    lat = np.deg2rad(lat_deg)
    dec = np.deg2rad(dec_deg)
    lam = C_LIGHT / freq_hz
    i, j = np.triu_indices(n_ant, k=1)
    b = (enu[j] - enu[i]) / lam                        # [nb][3] east, north, up (wavelengths)
    E, Nn, U = b[:, 0], b[:, 1], b[:, 2]
    X = -np.sin(lat) * Nn + np.cos(lat) * U
    Y = E
    Z = np.cos(lat) * Nn + np.sin(lat) * U
    H = np.linspace(-0.5 * hours, 0.5 * hours, n_dumps) * (2.0 * np.pi / 24.0)
    sH, cH = np.sin(H)[None, :], np.cos(H)[None, :]
    X, Y, Z = X[:, None], Y[:, None], Z[:, None]
    u = sH * X + cH * Y
    v = -np.sin(dec) * cH * X + np.sin(dec) * sH * Y + np.cos(dec) * Z
    w = np.cos(dec) * cH * X - np.cos(dec) * sH * Y + np.sin(dec) * Z
    uvw = np.stack([u.ravel(), v.ravel(), w.ravel()], axis=1)
    if max_vis is not None:
        uvw = uvw[:max_vis]
    return uvw


def scale_to_grid(uvw: np.ndarray, uv_limit: float) -> tuple[np.ndarray, float]:
    """Scale all coordinates by one factor s so that max(|u|, |v|) <= uv_limit; returns
    (scaled float32 uvw, s)."""
    m = float(np.abs(uvw[:, :2]).max())
    s = min(1.0, uv_limit / m)
    return (uvw * s).astype(np.float32), s


# --------------------------------------------------------------------------------------
# Workload shapes used by the tests and the benchmark
# --------------------------------------------------------------------------------------
def small_imaging(seed: int = 1, V: int = 20000):
    """Plain-method imaging problem: 256^2 image, 2 degree FOV, circular region of radius
    1 degree, |w| <= 500, (u, v) uniform in a disc of radius 2000, five point sources
    inside the circle with fluxes U(0.1, 1) Jy, unit weights, no noise."""
    N = 256
    dl = np.deg2rad(2.0) / N
    uvw = uniform_disc_uvw(V, 2000.0, 500.0, seed)
    sky = sources_in_disc(5, np.deg2rad(1.0), seed + 1)
    vis = predict(uvw, sky)
    return dict(N=N, cell_size=dl, uvw=uvw, vis=vis, sky=sky, weight=np.ones(V, dtype=np.float32))


def kernel_batch_planes(n_signed: int = 1024, w_lim: float = 20000.0, s_lo: int = 7, s_hi: int = 127):
    """Kernel-generation batch: signed w linearly spaced in [-w_lim, w_lim]; returns the
    distinct |w| values (ascending) and their supports, growing linearly with |w| from
    s_lo to s_hi: S = s_lo + round((s_hi - s_lo) |w| / w_lim)."""
    w = np.linspace(-w_lim, w_lim, n_signed)
    aw = np.unique(np.round(np.abs(w), 9))
    sup = (s_lo + np.rint((s_hi - s_lo) * aw / w_lim)).astype(np.int32)
    return w, aw, sup


def full_imaging(V: int = 1 << 23, seed: int = 3, n_sources: int = 200, noise_sigma: float = 1e-3,
                 N: int = 4096, fov_deg: float = 8.0, max_support: int = 127, predict_fn=None):
    """Full-imaging workload: 64 antennas in a 10 km disc, 8 h track at dec -30 (latitude
    -30), 1.4 GHz, uvw scaled so every footprint fits the 4096^2 grid, 200 sources in the
    circular FOV with log-uniform fluxes 1 mJy..1 Jy, Gaussian noise 1 mJy."""
    dl = np.deg2rad(fov_deg) / N
    du = 1.0 / (N * dl)
    n_dumps = -(-V // (64 * 63 // 2))
    uvw = track_uvw(n_dumps=n_dumps, seed=seed, max_vis=V)
    lim = (N / 2 - (max_support + 2)) * du
    uvw, s = scale_to_grid(uvw, lim)
    sky = sources_in_disc(n_sources, np.deg2rad(fov_deg / 2), seed + 1, 1e-3, 1.0, log_uniform=True)
    return dict(N=N, cell_size=dl, uvw=uvw, sky=sky, scale=s, noise_sigma=noise_sigma,
                noise_seed=seed + 2)


def batch_problems(n: int = 48, seed: int = 100, sizes=(512, 1024, 2048, 4096), planes=(32, 512),
                   vis=(100_000, 4_000_000), fov_deg: float = 8.0, n_sources: int = 20):
    """Independent imaging problems of uneven size: grid side drawn from `sizes`, plane count
    log-uniform in `planes`, visibility count log-uniform in `vis`; each generated like the
    full-imaging workload (64-antenna track at dec -30, uvw scaled to fit the grid) with its
    own seed.  Returns a list of dicts with N, cell_size, P, max_support, uvw, sky."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.choice(sizes))
        P = int(round(np.exp(rng.uniform(np.log(planes[0]), np.log(planes[1])))))
        V = int(round(np.exp(rng.uniform(np.log(vis[0]), np.log(vis[1])))))
        s_max = min(127, N // 8 - 1)
        dl = np.deg2rad(fov_deg) / N
        du = 1.0 / (N * dl)
        n_dumps = -(-V // (64 * 63 // 2))
        uvw = track_uvw(n_dumps=n_dumps, seed=seed + 7 * i + 1, max_vis=V)
        uvw, s = scale_to_grid(uvw, (N / 2 - (s_max + 2)) * du)
        sky = sources_in_disc(n_sources, np.deg2rad(fov_deg / 2), seed + 7 * i + 2, 1e-3, 1.0, log_uniform=True)
        out.append(dict(N=N, cell_size=dl, P=min(P, V), max_support=s_max, uvw=uvw, sky=sky, scale=s))
    return out
