"""Gradients of the differentiable visibility prediction (hand-written CUDA backward)
against FP64 central finite differences of the oracle's forward model, and against the
oracle's analytic image gradient (gridding is the adjoint of degridding)."""
import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import f32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problem(seed=0):
    N = 128
    dl = np.deg2rad(4.0) / N
    R, os_ = 256, 4
    planes = np.array([0.0, 150.0, 300.0, 450.0])
    sup = np.array([4, 5, 6, 8])
    g = o.Geometry(N, dl, os_, 8, 1, 0.0, R)
    du = g.du
    uvw = synth.uniform_disc_uvw(2000, (N / 2 - 10) * du, 450.0, seed + 1)
    rng = np.random.default_rng(seed)
    sky = synth.sources_in_disc(4, np.deg2rad(1.5), seed + 2)
    vobs = synth.predict(uvw, sky)
    wt = rng.uniform(0.5, 1.5, uvw.shape[0]).astype(np.float32)
    # smooth model image: a few Gaussian blobs, plus the tapered taper itself as parameters
    yy, xx = np.mgrid[0:N, 0:N] - N / 2
    img = np.zeros((N, N))
    for _ in range(5):
        cx, cy = rng.uniform(-30, 30, 2)
        img += rng.uniform(0.2, 1.0) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * rng.uniform(2, 6) ** 2))
    img = img.astype(np.float32)
    taper = synth.gaussian_taper_samples(N, dl, R, 0.25).astype(np.float32)
    return g, planes, sup, uvw, vobs, wt, img, taper


def _oracle_loss(g, planes, sup, uvw, vobs, wt, img, taper):
    v = o.predict_vis(g, img.astype(np.float64), taper.astype(np.float64), planes, sup, uvw)
    r = v - vobs.astype(np.complex128)
    return float(np.sum(wt.astype(np.float64) * (r.real ** 2 + r.imag ** 2))), v


def _gpu_grads(g, planes, sup, uvw, vobs, wt, img, taper, grid_method=3):
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.autograd import Predictor, chi2

    dev = torch.device("cuda")
    plan = wp.Plan(g.image_size, g.cell_size, g.oversampling, g.max_support, 1, 0.0, g.radial_samples,
                   grid_method=grid_method)
    pr = Predictor(plan, planes, sup, torch.tensor(uvw, device=dev))
    I = torch.tensor(img, device=dev, requires_grad=True)
    t = torch.tensor(taper, device=dev, requires_grad=True)
    vis = pr(I, t)
    L = chi2(vis, torch.tensor(vobs, device=dev), torch.tensor(wt, device=dev))
    L.backward()
    return float(L.detach()), vis.detach().cpu().numpy(), I.grad.cpu().numpy(), t.grad.cpu().numpy()


@pytest.mark.parametrize("grid_method", [3, 9])
def test_forward_prediction_matches_oracle(grid_method):
    """Prediction (degridding of the model image's grid) by the warp-per-visibility degridder
    (method 3's plan) and by the slot walk (method 9)."""
    g, planes, sup, uvw, vobs, wt, img, taper = _problem()
    L, vis, _, _ = _gpu_grads(g, planes, sup, uvw, vobs, wt, img, taper, grid_method)
    L0, v0 = _oracle_loss(g, planes, sup, uvw, vobs, wt, img, taper)
    assert np.abs(vis - v0).max() < 1e-4 * np.abs(v0).max()
    assert L == pytest.approx(L0, rel=1e-4)


@pytest.mark.parametrize("grid_method", [3, 9])
def test_image_gradient_matches_oracle_adjoint_and_finite_differences(grid_method):
    g, planes, sup, uvw, vobs, wt, img, taper = _problem(1)
    _, _, gI, _ = _gpu_grads(g, planes, sup, uvw, vobs, wt, img, taper, grid_method)
    # oracle analytic gradient: dL/dI = Re(A^H gv), gv = 2 wt (V - Vobs): grid(gv) then the
    # dirty-image map (both adjoints in the oracle)
    _, v0 = _oracle_loss(g, planes, sup, uvw, vobs, wt, img, taper)
    gv = 2.0 * wt.astype(np.float64) * (v0 - vobs.astype(np.complex128))
    ks = o.wkernels(g, taper.astype(np.float64), planes, supports=sup)
    b = o.bin_vis(g, uvw, planes, ks.support)
    Gg = o.grid(g, ks, b, gv.astype(np.complex64))   # unit weights, complex64 rounding of gv
    ref = o.dirty_image(g, Gg, taper.astype(np.float64), 1.0)
    assert np.abs(gI - ref).max() < 2e-4 * np.abs(ref).max()
    # FP64 central differences of the oracle's chi^2 on 64 random pixels inside the circle
    rng = np.random.default_rng(3)
    im_, il_ = np.nonzero(o.disc_mask(g))
    pick = rng.choice(im_.size, 64, replace=False)
    h = 1e-3
    for q in pick:
        a, bq = im_[q], il_[q]
        p = img.astype(np.float64).copy()
        p[a, bq] += h
        lp, _ = _oracle_loss(g, planes, sup, uvw, vobs, wt, p, taper)
        p[a, bq] -= 2 * h
        lm, _ = _oracle_loss(g, planes, sup, uvw, vobs, wt, p, taper)
        fd = (lp - lm) / (2 * h)
        assert abs(gI[a, bq] - fd) < 2e-3 * np.abs(ref).max() + 1e-3 * abs(fd), (a, bq, gI[a, bq], fd)


def test_taper_gradient_matches_finite_differences():
    """16 taper samples spread over the radius; the oracle recomputes the kernels (Hankel
    transform of the perturbed taper) and the image-to-grid division for each."""
    g, planes, sup, uvw, vobs, wt, img, taper = _problem(2)
    _, _, _, gt = _gpu_grads(g, planes, sup, uvw, vobs, wt, img, taper)
    idx = np.linspace(0, g.radial_samples - 1, 16).round().astype(int)
    fds = []
    for i in idx:
        h = 1e-4 * max(abs(float(taper[i])), 1e-3)
        tp = taper.astype(np.float64).copy()
        tp[i] += h
        lp, _ = _oracle_loss(g, planes, sup, uvw, vobs, wt, img, tp)
        tp[i] -= 2 * h
        lm, _ = _oracle_loss(g, planes, sup, uvw, vobs, wt, img, tp)
        fds.append((lp - lm) / (2 * h))
    fds = np.array(fds)
    scale = np.abs(fds).max()
    assert np.abs(gt[idx] - fds).max() < 5e-3 * scale, np.c_[gt[idx], fds]
