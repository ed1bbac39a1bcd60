"""GPU parity of kernel generation (screen, Hankel transform, truncation, spline, resample)
against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import KERNEL_TOL, f32, rel_l2, supports_match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _wp():
    import paper_1904_08463_gb300 as wp

    return wp


def _run(N, dl, os_, s_max, s_min, tau, R, interp, kernelgen, planes, supports=None, sigma=0.3):
    wp = _wp()
    dev = torch.device("cuda")
    plan = wp.Plan(N, dl, os_, s_max, s_min, tau, R, interp, kernelgen)
    g = o.Geometry(N, dl, os_, s_max, s_min, tau, R, 0 if interp == "cubic" else 1)
    taper = synth.gaussian_taper_samples(N, dl, R, sigma)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), planes, supports=supports)
    torch.cuda.synchronize()
    ks = o.wkernels(g, f32(taper), planes, supports=supports)
    return plan, g, wk, ks


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


@pytest.mark.parametrize("kernelgen", ["fp32", "tf32x3", "bf16x3", "bf16x6"])
def test_small_imaging_kernels(kernelgen):
    """256^2, 2 deg FOV, 16 |w|-planes <= 500, os 8, R 512, S_max 15, 1 % truncation."""
    N, dl = 256, np.deg2rad(2.0) / 256
    planes = np.linspace(0.0, 500.0, 16)
    plan, g, wk, ks = _run(N, dl, 8, 15, 3, 0.01, 512, "cubic", kernelgen, planes)
    _compare(g, wk, ks)


@pytest.mark.parametrize("kernelgen", ["fp32", "tf32x3", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("os_,R,P,interp", [(1, 300, 5, "cubic"), (4, 97, 3, "linear"),
                                            (16, 256, 70, "cubic"), (8, 2048, 130, "linear")])
def test_kernels_ragged_shapes(os_, R, P, interp, kernelgen):
    """Plane counts off the 64-column tile, R off the 32-deep slice, os 1 and 16, both
    interpolations, supports fixed by the caller (including the minimum 1)."""
    N, dl = 128, np.deg2rad(4.0) / 128
    planes = np.linspace(0.0, 1500.0, P)
    rng = np.random.default_rng(P)
    sup = rng.integers(1, 13, P)
    plan, g, wk, ks = _run(N, dl, os_, 12, 1, 0.0, R, interp, kernelgen, planes, supports=sup)
    _compare(g, wk, ks)


@pytest.mark.parametrize("kernelgen", ["fp32", "tf32x3", "bf16x3", "bf16x6"])
def test_large_w_kernels_sampled(kernelgen):
    """1024 signed planes linspace[-20000, 20000] (512 distinct |w|), R 4096, os 8,
    supports 7..127 growing with |w|, 8 degree FOV on 4096^2: every plane is generated
    on the GPU; 6 planes spread over |w| are checked against the oracle."""
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R = 4096, np.deg2rad(8.0) / 4096, 4096
    _, aw, sup = synth.kernel_batch_planes()
    plan = wp.Plan(N, dl, 8, 127, 7, 0.0, R, "cubic", kernelgen)
    taper = synth.gaussian_taper_samples(N, dl, R)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), aw, supports=sup)
    torch.cuda.synchronize()
    g = o.Geometry(N, dl, 8, 127, 7, 0.0, R)
    pick = [0, 100, 255, 300, 470, 511]
    ks = o.wkernels(g, f32(taper), aw[pick], supports=sup[pick])
    radial = wk.radial.cpu().numpy()
    off = wk.offsets.cpu().numpy()
    for j, p in enumerate(pick):
        e = rel_l2(radial[p], ks.radial[j])
        assert e < KERNEL_TOL, f"|w| = {aw[p]:.1f}: radial rel. L2 {e:.3e}"
        c = wk.cache[int(off[p]):int(off[p + 1])].cpu().numpy()
        e = rel_l2(c, ks.cache[ks.offsets[j]:ks.offsets[j + 1]])
        assert e < KERNEL_TOL, f"|w| = {aw[p]:.1f}: cache rel. L2 {e:.3e}"


def test_tensor_core_route_matches_fp32_route_on_every_plane():
    """All 512 planes of the large-|w| batch: the tcgen05 TF32x3 and BF16x6 radial lines agree
    with the FP32 SIMT ones to well inside the kernel tolerance (all are ~1e-7 from FP64;
    the six-product BF16 split keeps all 24 bits of the FP32 operands)."""
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R = 4096, np.deg2rad(8.0) / 4096, 4096
    _, aw, sup = synth.kernel_batch_planes()
    taper = torch.tensor(synth.gaussian_taper_samples(N, dl, R), dtype=torch.float32, device=dev)
    w = torch.tensor(aw, dtype=torch.float64, device=dev)
    out = {}
    for kg in ("fp32", "tf32x3", "bf16x6"):
        plan = wp.Plan(N, dl, 8, 127, 7, 0.0, R, "cubic", kg)
        ws = wp.kernelgen_prepare(plan, len(aw))
        out[kg] = wp.hankel_radial(plan, taper, w, ws)[0].cpu().numpy()
    den = np.linalg.norm(out["fp32"], axis=1)
    for kg in ("tf32x3", "bf16x6"):
        num = np.linalg.norm(out["fp32"] - out[kg], axis=1)
        assert (num / den).max() < 2e-6, kg


@pytest.mark.parametrize("os_,interp", [(3, "cubic"), (5, "linear"), (8, "cubic")])
def test_resample_staged_rows_odd_os_unaligned_cache(os_, interp):
    """Supports up to 60 (121-wide rows: several staged chunks per sub-kernel), odd and even
    oversampling, and a cache that starts 8 bytes past a 16-byte boundary: every plane
    against the oracle, and the mirror identities of the cache hold bit for bit
    (tap (jx, jy) of sub-kernel fu equals tap (2S + [fu > 0] - jx, jy) of (os - fu) mod os)."""
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R, s_max = 256, np.deg2rad(3.0) / 256, 512, 60
    planes = np.array([0.0, 150.0, 400.0, 900.0, 1400.0, 2000.0])
    sup = np.array([1, 2, 17, 33, 60, 59])
    plan = wp.Plan(N, dl, os_, s_max, 1, 0.0, R, interp, "tf32x3")
    taper = synth.gaussian_taper_samples(N, dl, R)
    w = torch.tensor(planes, dtype=torch.float64, device=dev)
    ws = wp.kernelgen_prepare(plan, len(planes))
    radial, spline_m, _ = wp.hankel_radial(plan, torch.tensor(taper, dtype=torch.float32, device=dev), w, ws)
    off = wp.kernel_layout(plan, sup.tolist())
    store = torch.full((off[-1] + 2,), float("nan"), dtype=torch.complex64, device=dev)
    cache = store[1:off[-1] + 1]
    assert cache.data_ptr() % 16 == 8
    wp.resample(plan, radial, spline_m, torch.tensor(sup, dtype=torch.int32, device=dev),
                torch.tensor(off, dtype=torch.int64, device=dev), cache)
    torch.cuda.synchronize()
    got = store.cpu().numpy()
    assert np.isnan(got[0].real) and np.isnan(got[-1].real), "wrote outside the cache"
    got = got[1:-1]
    g = o.Geometry(N, dl, os_, s_max, 1, 0.0, R, 0 if interp == "cubic" else 1)
    ks = o.wkernels(g, f32(taper), planes, supports=sup)
    for p, S in enumerate(sup):
        c = got[off[p]:off[p + 1]]
        e = rel_l2(c, ks.cache[ks.offsets[p]:ks.offsets[p + 1]])
        assert e < KERNEL_TOL, f"plane {p} (S = {S}): cache rel. L2 {e:.3e}"
        Wd = 2 * S + 1
        k = c.reshape(os_, os_, Wd, Wd)           # [fv][fu][jy][jx]
        for fu in range(os_):
            fu2, sh = ((os_ - fu) % os_, 1 if fu else 0)
            jx = np.arange(sh, Wd)
            mj = 2 * S + sh - jx
            assert np.array_equal(k[:, fu][..., jx].view(np.uint64), k[:, fu2][..., mj].view(np.uint64))
            if fu:
                assert not np.any(k[:, fu][..., 0])


@pytest.mark.parametrize("kernelgen", ["tf32x3", "bf16x3", "bf16x6", "projslice"])
def test_prolate_taper_kernels(kernelgen):
    """The radially symmetric prolate spheroidal taper (c = 3 pi) instead of the Gaussian:
    the small imaging geometry's kernels against the oracle, by both Hankel routes."""
    pytest.importorskip("scipy.special")
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R = 256, np.deg2rad(2.0) / 256, 512
    planes = np.linspace(0.0, 500.0, 16)
    plan = wp.Plan(N, dl, 8, 15, 3, 0.01, R, "cubic", kernelgen)
    g = o.Geometry(N, dl, 8, 15, 3, 0.01, R)
    taper = synth.pswf_taper_samples(N, dl, R)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), planes)
    torch.cuda.synchronize()
    ks = o.wkernels(g, f32(taper), planes, route="hankel" if kernelgen != "projslice" else "projslice")
    _compare(g, wk, ks)


def test_resample_largest_support():
    """Support 511 at os 8, the largest the plan allows: the staged line (64 KB) and four
    regions of one 1023-tap row leave room for one resample block per SM, one row per chunk
    -- the cache against the oracle."""
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R = 1024, np.deg2rad(4.0) / 1024, 1024
    planes = np.array([0.0, 3000.0])
    sup = np.array([511, 200])
    plan = wp.Plan(N, dl, 8, 511, 1, 0.0, R, "cubic", "tf32x3")
    taper = synth.gaussian_taper_samples(N, dl, R)
    wk = wp.make_wkernels(plan, torch.tensor(taper, dtype=torch.float32, device=dev), planes, supports=sup)
    torch.cuda.synchronize()
    g = o.Geometry(N, dl, 8, 511, 1, 0.0, R)
    ks = o.wkernels(g, f32(taper), planes, supports=sup)
    off = wk.offsets.cpu().numpy()
    for p in range(len(planes)):
        c = wk.cache[int(off[p]):int(off[p + 1])].cpu().numpy()
        e = rel_l2(c, ks.cache[ks.offsets[p]:ks.offsets[p + 1]])
        assert e < KERNEL_TOL, f"plane {p} (S = {sup[p]}): cache rel. L2 {e:.3e}"


@pytest.mark.parametrize("kernelgen", ["tf32x3", "bf16x3", "bf16x6", "projslice"])
def test_every_radial_line_of_the_512_plane_batch(kernelgen):
    """All 512 radial lines of the headline batch (R 4096, K_out 1152, |w| to 20000) against
    the FP64 oracle, each within the kernel tolerance (the caches are sampled elsewhere)."""
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R = 4096, np.deg2rad(8.0) / 4096, 4096
    _, aw, sup = synth.kernel_batch_planes()
    plan = wp.Plan(N, dl, 8, 127, 7, 0.0, R, "cubic", kernelgen)
    taper = synth.gaussian_taper_samples(N, dl, R)
    ws = wp.kernelgen_prepare(plan, len(aw))
    radial, _, _ = wp.hankel_radial(plan, torch.tensor(taper, dtype=torch.float32, device=dev),
                                    torch.tensor(aw, dtype=torch.float64, device=dev), ws)
    radial = radial.cpu().numpy()
    g = o.Geometry(N, dl, 8, 127, 7, 0.0, R)
    ks = o.wkernels(g, f32(taper), aw, supports=sup, with_cache=False,
                    route="hankel" if kernelgen != "projslice" else "projslice")
    errs = np.array([rel_l2(radial[p], ks.radial[p]) for p in range(len(aw))])
    assert errs.max() < KERNEL_TOL, f"worst plane {errs.argmax()}: {errs.max():.3e}"


def test_one_prepared_workspace_serves_every_route():
    """The workspace layout and tables do not depend on plan.kernelgen: a workspace prepared
    under one route gives every other route the same radial lines, bit for bit, as a
    workspace prepared under that route."""
    wp = _wp()
    dev = torch.device("cuda")
    N, dl, R = 256, np.deg2rad(2.0) / 256, 512
    planes = torch.tensor(np.linspace(0.0, 500.0, 16), dtype=torch.float64, device=dev)
    taper = torch.tensor(synth.gaussian_taper_samples(N, dl, R), dtype=torch.float32, device=dev)
    base = wp.Plan(N, dl, 8, 15, 3, 0.0, R, "cubic", "tf32x3")
    shared = wp.kernelgen_prepare(base, 16)
    for kg in ("fp32", "tf32x3", "bf16x3", "bf16x6", "projslice"):
        plan = base.replace(kernelgen=kg)
        own = wp.kernelgen_prepare(plan, 16)
        a = wp.hankel_radial(plan, taper, planes, shared)[0].cpu().numpy()
        b = wp.hankel_radial(plan, taper, planes, own)[0].cpu().numpy()
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), kg
