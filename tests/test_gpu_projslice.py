"""GPU parity of the projection-slice Hankel route (Section 4.3.1, Alg. 2 steps 4-12):
workspace image projected onto one axis, zero-padded by os, batched 1D cuFFT, then the same
truncation, spline and resample as the matrix route -- against the FP64 oracle's projection
route on the same seeded inputs."""
import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import KERNEL_TOL, f32, rel_l2, supports_match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run(N, dl, os_, s_max, s_min, tau, R, interp, planes, supports=None, sigma=0.3):
    import paper_1904_08463_gb300 as wp

    dev = torch.device("cuda")
    plan = wp.Plan(N, dl, os_, s_max, s_min, tau, R, interp, "projslice")
    g = o.Geometry(N, dl, os_, s_max, s_min, tau, R, 0 if interp == "cubic" else 1)
    taper = synth.gaussian_taper_samples(N, dl, R, sigma)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), planes, supports=supports)
    torch.cuda.synchronize()
    ks = o.wkernels(g, f32(taper), planes, supports=supports, route="projslice")
    return g, wk, ks


def _compare(g, wk, ks, tol=KERNEL_TOL):
    radial = wk.radial.cpu().numpy()
    for p in range(len(ks.w_planes)):
        e = rel_l2(radial[p], ks.radial[p])
        assert e < tol, f"plane {p} (|w| = {ks.w_planes[p]}): radial rel. L2 {e:.3e}"
    sup = wk.support.cpu().numpy()
    assert supports_match(sup, ks.radial, ks.support, g.trunc_frac, g.oversampling)
    cache = wk.cache.cpu().numpy()
    off = wk.offsets.cpu().numpy()
    for p in range(len(ks.w_planes)):
        if sup[p] != ks.support[p]:
            continue
        e = rel_l2(cache[off[p]:off[p + 1]], ks.cache[ks.offsets[p]:ks.offsets[p + 1]])
        assert e < tol, f"plane {p}: cache rel. L2 {e:.3e}"


def test_projslice_small_imaging_kernels():
    """256^2, 2 deg FOV, 16 |w|-planes <= 500, os 8, R 512, S_max 15, 1 % truncation."""
    N, dl = 256, np.deg2rad(2.0) / 256
    g, wk, ks = _run(N, dl, 8, 15, 3, 0.01, 512, "cubic", np.linspace(0.0, 500.0, 16))
    _compare(g, wk, ks)


@pytest.mark.parametrize("os_,R,P,interp", [(1, 300, 5, "cubic"), (3, 97, 3, "linear"),
                                            (16, 256, 70, "cubic"), (5, 2048, 33, "linear")])
def test_projslice_ragged_shapes(os_, R, P, interp):
    """Odd and large oversampling (line length M os from 32 to 512), both interpolations,
    plane counts off any tile, supports fixed by the caller (including the minimum 1)."""
    N, dl = 128, np.deg2rad(4.0) / 128
    planes = np.linspace(0.0, 1500.0, P)
    sup = np.random.default_rng(P).integers(1, 13, P)
    g, wk, ks = _run(N, dl, os_, 12, 1, 0.0, R, interp, planes, supports=sup)
    _compare(g, wk, ks)


def test_projslice_large_w_sampled():
    """The 512-plane batch (|w| to 20000, R 4096, os 8, supports 7..127 by |w|, 8 degrees on
    4096^2, workspace M = 256, line length 2048): every plane on the GPU, 6 spread over |w|
    checked against the oracle."""
    import paper_1904_08463_gb300 as wp

    dev = torch.device("cuda")
    N, dl, R = 4096, np.deg2rad(8.0) / 4096, 4096
    _, aw, sup = synth.kernel_batch_planes()
    plan = wp.Plan(N, dl, 8, 127, 7, 0.0, R, "cubic", "projslice")
    taper = synth.gaussian_taper_samples(N, dl, R)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), aw, supports=sup)
    torch.cuda.synchronize()
    g = o.Geometry(N, dl, 8, 127, 7, 0.0, R)
    pick = [0, 100, 255, 300, 470, 511]
    ks = o.wkernels(g, f32(taper), aw[pick], supports=sup[pick], route="projslice")
    radial = wk.radial.cpu().numpy()
    off = wk.offsets.cpu().numpy()
    for j, p in enumerate(pick):
        e = rel_l2(radial[p], ks.radial[j])
        assert e < KERNEL_TOL, f"|w| = {aw[p]:.1f}: radial rel. L2 {e:.3e}"
        c = wk.cache[int(off[p]):int(off[p + 1])].cpu().numpy()
        e = rel_l2(c, ks.cache[ks.offsets[j]:ks.offsets[j + 1]])
        assert e < KERNEL_TOL, f"|w| = {aw[p]:.1f}: cache rel. L2 {e:.3e}"
