"""GPU parity of the standard 2D-FFT kernel generation (Alg. 1 with workspace
undersampling, Section 4.2) against the oracle's numpy-FFT route, and agreement of the two
GPU routes (2D FFT and Hankel) on a radially smooth input (Section 4.3)."""
import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import KERNEL_TOL, f32, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wp():
    import paper_1904_08463_gb300 as wp

    return wp


@pytest.mark.parametrize("circular", [True, False])
def test_fft_route_matches_oracle_small(circular):
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R, os_ = 128, np.deg2rad(4.0) / 128, 512, 8
    plan = wp.Plan(N, dl, os_, 12, 1, 0.0, R)
    g = o.Geometry(N, dl, os_, 12, 1, 0.0, R)
    taper = synth.gaussian_taper_samples(N, dl, R)
    planes = np.array([0.0, 150.0, 700.0, 1500.0, 3000.0])
    sup = np.array([3, 5, 8, 12, 12])
    wk = wp.fft_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), planes, sup, circular)
    off = wk.offsets.cpu().numpy()
    cache = wk.cache.cpu().numpy()
    for p, (w, s) in enumerate(zip(planes, sup)):
        ref = o.fft_wkernel(g, f32(taper), w, int(s), circular=circular).ravel()
        e = rel_l2(cache[off[p]:off[p + 1]], ref)
        assert e < KERNEL_TOL, f"|w| = {w}: rel. L2 {e:.3e}"


def test_fft_route_matches_oracle_large_workspace():
    """The kernel batch's geometry: M = 256 workspace, 2048^2 padded transform."""
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R = 4096, np.deg2rad(8.0) / 4096, 4096
    _, aw, sup = synth.kernel_batch_planes()
    pick = [3, 400]
    plan = wp.Plan(N, dl, 8, 127, 7, 0.0, R)
    g = o.Geometry(N, dl, 8, 127, 7, 0.0, R)
    taper = synth.gaussian_taper_samples(N, dl, R)
    wk = wp.fft_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), aw[pick], sup[pick])
    off = wk.offsets.cpu().numpy()
    cache = wk.cache.cpu().numpy()
    for j, p in enumerate(pick):
        ref = o.fft_wkernel(g, f32(taper), aw[p], int(sup[p])).ravel()
        e = rel_l2(cache[off[j]:off[j + 1]], ref)
        assert e < KERNEL_TOL, f"|w| = {aw[p]:.1f}: rel. L2 {e:.3e}"


def test_fft_and_hankel_routes_agree_on_smooth_radial_input():
    """Narrow Gaussian taper that vanishes well inside the disc: the two GPU routes compute
    the same kernels to the discretisation error pinned for the oracle (< 5e-6)."""
    wp = _wp()
    dev = torch.device("cuda")
    N, r_max, R = 64, 0.02, 4096
    dl = 2 * r_max / N
    a = 40.0 / r_max ** 2
    r = (np.arange(R) + 0.5) * r_max / R
    taper = torch.tensor(np.exp(-a * r * r), dtype=torch.float32, device=dev)
    planes = np.array([0.0, 20000.0])
    sup = [10, 10]
    for kg in ("fp32", "tf32x3"):
        plan = wp.Plan(N, dl, 8, 15, 3, 0.0, R, "cubic", kg)
        hk = wp.make_wkernels(plan, taper, planes, supports=sup).cache.cpu().numpy()
        fk = wp.fft_wkernels(plan, taper, planes, sup).cache.cpu().numpy()
        assert rel_l2(fk, hk) < 1e-5
