"""Dirty images of the benchmark's own imaging step against the FP64 oracle.

The step under test is ``Imager.step`` -- the one ``bench.py`` times: plane values on the
device (Alg. 2 steps 1-3), Hankel kernels by the tensor-core BF16x3 route with supports chosen
by the 1 % truncation rule on the device (Section 3.1) into the maximum-support cache layout,
the gridder shape the autotuner picks for the problem, and the dirty image normalised by the
weight sum read on the device (Section 3).  The oracle computes the same image from the same
inputs in FP64 (its own plane values, radial lines, supports, cache, gridding and transform);
the two are compared pixel by pixel inside the circle where the image is defined (Section 6),
to 1e-4 of the peak."""
import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import IMAGE_TOL, f32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _full_imaging_subset(n=65536, seed=12):
    """A seeded subset of the full-imaging workload's visibilities (8M-visibility track set,
    same geometry, sky and noise recipe), values by direct evaluation of Eq. 2."""
    d = synth.full_imaging()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(d["uvw"].shape[0], n, replace=False))
    uvw = np.ascontiguousarray(d["uvw"][idx])
    vis = synth.add_noise(synth.predict(uvw, d["sky"]), d["noise_sigma"], d["noise_seed"])
    return d["N"], d["cell_size"], uvw, vis


def _oracle_image(N, dl, R, P, uvw, vis, wt=None, s_max=127, taper=None):
    g = o.Geometry(N, dl, 8, s_max, 3, 0.01, R)
    tap = f32(taper if taper is not None else synth.gaussian_taper_samples(N, dl, R))
    planes = o.mean_w_planes(uvw[:, 2].astype(np.float64), P)
    ks = o.wkernels(g, tap, planes)
    b = o.bin_vis(g, uvw, planes, ks.support)
    keep = b.drop == 0
    wsum = float(np.sum(wt[keep].astype(np.float64))) if wt is not None else float(keep.sum())
    img = o.dirty_image(g, o.grid(g, ks, b, vis, wt), tap, wsum)
    return g, ks, b, img


_ORACLE = {}


def _subset_and_oracle():
    """The subset and the oracle's image of it, computed once for every gridder below."""
    if not _ORACLE:
        N, dl, uvw, vis = _full_imaging_subset()
        _ORACLE["inputs"] = (N, dl, uvw, vis)
        _ORACLE["oracle"] = _oracle_image(N, dl, 512, 512, uvw, vis)
    return _ORACLE["inputs"], _ORACLE["oracle"]


@pytest.mark.parametrize("shape", [None, (9, 64)])
def test_full_imaging_subset_through_the_benchmark_step(shape):
    """shape None: the gridder the autotuner picks for the subset; otherwise that gridder (the
    slot gridder, which the full-size benchmark picks) in the same step."""
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.imager import Imager

    dev = torch.device("cuda")
    (N, dl, uvw, vis), (g, ks, b, ref) = _subset_and_oracle()
    R, P = 512, 512
    plan = wp.Plan(N, dl, 8, 127, 3, 0.01, R, "cubic", "bf16x3")
    taper = synth.gaussian_taper_samples(N, dl, R)
    tap_d = torch.tensor(taper, dtype=torch.float32, device=dev)
    u_d = torch.tensor(uvw, device=dev).reshape(-1)
    v_d = torch.tensor(vis, device=dev)
    im = Imager(plan, tap_d, u_d, P)
    im.autotune(u_d, v_d, choices=None if shape is None else [list(shape)])
    img = im.step(u_d, v_d).cpu().numpy()
    stats = im.stats.cpu().numpy()
    # the device's plane values and 1 % supports are the oracle's
    assert np.allclose(im.w_planes.cpu().numpy(), ks.w_planes, rtol=1e-13, atol=0)
    assert np.array_equal(im.support.cpu().numpy(), ks.support)
    assert stats[1] == (b.drop != 0).sum() and stats[0] == float((b.drop == 0).sum())
    inside = o.disc_mask(g)
    err = np.abs(img - ref)[inside].max() / np.abs(ref).max()
    assert err <= IMAGE_TOL, f"max error {err:.3e} of peak (gridder {im.plan.grid_method},{im.plan.grid_tile})"
    assert np.all(img[~inside] == 0)


@pytest.mark.parametrize("kernelgen", ["fp32", "tf32x3", "bf16x3", "bf16x6", "projslice"])
def test_small_imaging_every_kernel_route(kernelgen):
    """The small imaging problem (20k visibilities, 5 sources, 16 planes, S 5) with the
    kernels of each route -- FP32 SIMT, the three tensor-core split routes, projection-slice --
    gridded and imaged on the device, against the oracle's image of the same route."""
    import paper_1904_08463_gb300 as wp

    dev = torch.device("cuda")
    d = synth.small_imaging()
    N, dl, R = d["N"], d["cell_size"], 512
    planes = np.linspace(0.0, 500.0, 16)
    sup = np.full(16, 5)
    plan = wp.Plan(N, dl, 8, 15, 1, 0.0, R, "cubic", kernelgen)
    g = o.Geometry(N, dl, 8, 15, 1, 0.0, R)
    taper = synth.gaussian_taper_samples(N, dl, R)
    tap_d = torch.tensor(taper, dtype=torch.float32, device=dev)
    wk = wp.make_wkernels(plan, tap_d, planes, supports=sup)
    ks = o.wkernels(g, f32(taper), planes, supports=sup, route="projslice" if kernelgen == "projslice" else "hankel")
    G, stats = wp.grid(plan, wk, torch.tensor(d["uvw"], device=dev).reshape(-1), torch.tensor(d["vis"], device=dev),
                       torch.tensor(d["weight"], device=dev))
    img = wp.dirty_image(plan, tap_d, G, stats).cpu().numpy()
    b = o.bin_vis(g, d["uvw"], planes, sup)
    ref = o.dirty_image(g, o.grid(g, ks, b, d["vis"], d["weight"]), f32(taper),
                        float(d["weight"][b.drop == 0].sum()))
    assert np.abs(img - ref).max() < IMAGE_TOL * np.abs(ref).max()
    assert np.all(img[~o.disc_mask(g)] == 0)
