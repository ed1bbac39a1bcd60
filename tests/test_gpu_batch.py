"""Batched uneven imaging problems: the graph-replayed batch gives the same dirty images as
running the problems one at a time, as the plain API calls and as the FP64 oracle; the
autotuner's choices do not change results; weights and dropped visibilities normalise the
images by the weights actually gridded."""
import numpy as np
import pytest

import synth
from oracle import oracle as o
from tests.common import IMAGE_TOL, f32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problems(dev, n=5, seed=7, uv_scale=1.0, weights=False, vis_range=(2000, 60000)):
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.batch import Problem

    specs = synth.batch_problems(n=n, seed=seed, sizes=(256, 512), planes=(8, 40), vis=vis_range)
    out = []
    for i, d in enumerate(specs):
        R = 256
        d["uvw"] = (d["uvw"] * np.float32(uv_scale)).astype(np.float32)
        d["vis"] = synth.predict(d["uvw"], d["sky"])
        d["wt"] = (np.random.default_rng(seed + i).uniform(0.3, 2.0, d["uvw"].shape[0]).astype(np.float32)
                   if weights else None)
        plan = wp.Plan(d["N"], d["cell_size"], 8, d["max_support"], 3, 0.01, R, "cubic", "fp32")
        taper = torch.tensor(synth.gaussian_taper_samples(d["N"], d["cell_size"], R), dtype=torch.float32,
                             device=dev)
        uvw = torch.tensor(d["uvw"], device=dev).reshape(-1)
        vis = torch.tensor(d["vis"], device=dev)
        wt = torch.tensor(d["wt"], device=dev) if weights else None
        out.append(Problem(plan, taper, uvw, vis, d["P"], wt))
    return specs, out


def _oracle_image(d, R=256):
    """The oracle's dirty image of one batch problem: its own plane values (means of
    equal-count |w| chunks), FP64 kernels with its own 1 % supports, gridding and image,
    normalised by the weights of the visibilities it kept."""
    N, dl = d["N"], d["cell_size"]
    g = o.Geometry(N, dl, 8, d["max_support"], 3, 0.01, R)
    tap = f32(synth.gaussian_taper_samples(N, dl, R))
    planes = o.mean_w_planes(d["uvw"][:, 2].astype(np.float64), d["P"])
    ks = o.wkernels(g, tap, planes)
    b = o.bin_vis(g, d["uvw"], planes, ks.support)
    keep = b.drop == 0
    wsum = float(np.sum(d["wt"][keep].astype(np.float64))) if d["wt"] is not None else float(keep.sum())
    return g, ks, b, wsum, o.dirty_image(g, o.grid(g, ks, b, d["vis"], d["wt"]), tap, wsum)


def test_graph_batch_matches_sequential_and_direct_calls(tmp_path):
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.autotune import Autotuner
    from paper_1904_08463_gb300.batch import BatchImager

    dev = torch.device("cuda")
    specs, pbs = _problems(dev)
    tuner = Autotuner(str(tmp_path / "tune.json"))
    b = BatchImager(pbs, n_streams=3, tuner=tuner)
    b.run_sequential()
    torch.cuda.synchronize()
    seq = [im.cpu().numpy().copy() for im in b.images]
    assert b.dropped() == 0
    b.replay()
    b.replay()
    torch.cuda.synchronize()
    rep = [im.cpu().numpy() for im in b.images]
    for a, c in zip(seq, rep):
        assert np.abs(a - c).max() <= 1e-5 * np.abs(a).max()
    # plain API calls, default launch shapes, on problem 0
    pb = pbs[0]
    st = b.states[0]
    wk = wp.make_wkernels(pb.plan.replace(trunc_frac=0.0), pb.taper, st.w_planes.cpu().numpy(),
                          supports=st.support.cpu().tolist())
    G, stats = wp.grid(pb.plan.replace(trunc_frac=0.0), wk, pb.uvw, pb.vis)
    img = wp.dirty_image(pb.plan, pb.taper, G, float(stats[0].item())).cpu().numpy()
    assert np.abs(img - seq[0]).max() <= 1e-5 * np.abs(img).max()
    assert len(tuner.table) >= 2
    # the replayed images against the FP64 oracle, problem by problem (routes and gridder
    # shapes as the autotuner picked them)
    for i in range(len(pbs)):
        g, ks, bo, wsum, ref = _oracle_image(specs[i])
        assert np.array_equal(b.states[i].support.cpu().numpy(), ks.support), i
        assert np.abs(rep[i] - ref).max() <= IMAGE_TOL * np.abs(ref).max(), i


def test_graph_batch_of_large_grids_matches_sequential():
    """Grids of 2048^2 and 4096^2, whose cuFFT plans carry work areas: the library keeps one
    plan per stream, so the graph's concurrent branches never share a work area, and the
    imager creates those plans in an uncaptured pass on the capture's own streams."""
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.batch import BatchImager, Problem

    dev = torch.device("cuda")
    specs = synth.batch_problems(n=3, seed=11, sizes=(2048, 4096), planes=(8, 16), vis=(5000, 20000))
    pbs = []
    for d in specs:
        R = 256
        plan = wp.Plan(d["N"], d["cell_size"], 8, d["max_support"], 3, 0.01, R, "cubic", "tf32x3", 64, 3)
        taper = torch.tensor(synth.gaussian_taper_samples(d["N"], d["cell_size"], R), dtype=torch.float32,
                             device=dev)
        uvw = torch.tensor(d["uvw"], device=dev).reshape(-1)
        vis = torch.tensor(synth.predict(d["uvw"], d["sky"]), device=dev)
        pbs.append(Problem(plan, taper, uvw, vis, d["P"]))
    b = BatchImager(pbs, n_streams=3)
    b.run_sequential()
    torch.cuda.synchronize()
    seq = [im.cpu().numpy().copy() for im in b.images]
    for _ in range(3):
        b.replay()
    torch.cuda.synchronize()
    for a, c in zip(seq, [im.cpu().numpy() for im in b.images]):
        assert np.abs(a - c).max() <= 1e-5 * np.abs(a).max()


def test_batch_normalises_by_the_weights_actually_gridded():
    """Non-unit weights and visibilities whose footprints leave the grid (dropped): every
    batched image equals wp_dirty_image of the same grid with the true sum of gridded weights
    (read back here), and the oracle's image (Section 3: weighted mean of the gridded data)."""
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.batch import BatchImager

    dev = torch.device("cuda")
    specs, pbs = _problems(dev, n=3, seed=17, uv_scale=1.6, weights=True)
    b = BatchImager(pbs, n_streams=2)
    assert b.dropped() > 0
    b.replay()
    b.replay()
    torch.cuda.synchronize()
    for i, (d, st) in enumerate(zip(specs, b.states)):
        img = st.image.cpu().numpy()
        g, ks, bo, wsum, ref = _oracle_image(d)
        assert np.array_equal(st.support.cpu().numpy(), ks.support), i
        stats = st.stats.cpu().numpy()
        assert stats[1] == (bo.drop != 0).sum() > 0, i
        assert stats[0] == pytest.approx(wsum, rel=1e-6), i
        G, _ = wp.grid(st.plan, st.wk, pbs[i].uvw, pbs[i].vis, pbs[i].weight)
        host = wp.dirty_image(st.plan, pbs[i].taper, G, float(stats[0])).cpu().numpy()
        assert np.abs(img - host).max() <= 1e-5 * np.abs(host).max(), i
        assert np.abs(img - ref).max() <= IMAGE_TOL * np.abs(ref).max(), i


def test_persistent_batch_matches_per_problem_gridding_and_the_oracle():
    """The persistent multi-problem gridder (one device queue for every problem's scatter and
    (plane, tile) items: a launch for the orderings, one for the items) against each problem's
    own wp_grid and, for the images, the oracle; replayed from a CUDA graph."""
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.batch import BatchImager

    dev = torch.device("cuda")
    specs, pbs = _problems(dev, n=5, seed=31, uv_scale=1.3, weights=True)
    b = BatchImager(pbs, n_streams=2, persistent=True)
    assert b.status() == 0
    b.replay()
    b.replay()
    torch.cuda.synchronize()
    assert b.status() == 0
    assert b.dropped() > 0
    for i, (d, st) in enumerate(zip(specs, b.states)):
        G, stats = wp.grid(st.plan.replace(grid_method=3, grid_tile=64), st.wk, pbs[i].uvw, pbs[i].vis,
                           pbs[i].weight)
        assert np.allclose(st.stats.cpu().numpy(), stats.cpu().numpy(), rtol=1e-9), i
        host = wp.dirty_image(st.plan, pbs[i].taper, G, float(stats[0].item())).cpu().numpy()
        img = st.image.cpu().numpy()
        assert np.abs(img - host).max() <= 1e-5 * np.abs(host).max(), i
        g, ks, bo, wsum, ref = _oracle_image(d)
        assert np.array_equal(st.support.cpu().numpy(), ks.support), i
        assert np.abs(img - ref).max() <= IMAGE_TOL * np.abs(ref).max(), i


def _jobs(dev, methods, seed, vis_range=(2000, 6000)):
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300 import api

    specs, pbs = _problems(dev, n=len(methods), seed=seed, vis_range=vis_range, weights=True, uv_scale=1.2)
    jobs, refs = [], []
    for d, pb, m in zip(specs, pbs, methods):
        plan = pb.plan.replace(trunc_frac=0.0, grid_method=m, grid_tile=64)
        planes = o.mean_w_planes(d["uvw"][:, 2].astype(np.float64), d["P"])
        wk = wp.make_wkernels(plan, pb.taper, planes, supports=[min(9, d["max_support"])] * d["P"])
        ws = wp.workspace(wp.grid_workspace_bytes(plan, wk.P, pb.vis.numel()), dev)
        G = torch.zeros((plan.image_size, plan.image_size), dtype=torch.complex64, device=dev)
        jobs.append(api.GridJob(plan, wk, pb.uvw, pb.vis, pb.weight, G, ws,
                                torch.zeros(2, dtype=torch.float64, device=dev)))
        refs.append([x.cpu().numpy() for x in wp.grid(plan.replace(grid_method=3), wk, pb.uvw, pb.vis, pb.weight)])
    return jobs, refs


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("methods", [(9, 9, 9), (3, 9, 3, 9), (9,)])
def test_persistent_batch_with_slot_jobs_matches_per_job_gridding(methods, fused):
    """Slot jobs (grid_method 9) -- alone or mixed with row-owned ones -- in the persistent
    launches: the gathers order each slot job's records before its items run (in a launch of
    their own, or fused: in the same launch, the items waiting for them); every grid and its
    stats equal the job's own wp_grid, twice in a row."""
    from paper_1904_08463_gb300 import api

    dev = torch.device("cuda")
    jobs, refs = _jobs(dev, methods, seed=53)
    bws = api.grid_batch_workspace(dev)
    for _ in range(2):
        for j in jobs:
            j.grid.zero_()
            j.stats.zero_()
        api.grid_batch(jobs, bws, fused=fused)
        torch.cuda.synchronize()
        assert api.grid_batch_status(bws) == 0
        for j, (G, st) in zip(jobs, refs):
            assert np.abs(j.grid.cpu().numpy() - G).max() <= 1e-5 * np.abs(G).max()
            assert np.allclose(j.stats.cpu().numpy(), st, rtol=1e-9)


@pytest.mark.parametrize("methods", [(3, 3), (9, 3)])
def test_persistent_batch_bounded_wait_expires_and_context_survives(methods):
    """With the record ordering (scatter / gather) withheld every gridding item's wait runs out:
    the batch status is WP_ERR_TIMEOUT, no grid cell is written, and the same context then grids
    correctly."""
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300 import api

    dev = torch.device("cuda")
    specs, pbs = _problems(dev, n=len(methods), seed=41, vis_range=(2000, 6000))
    jobs, refs = [], []
    for d, pb, m in zip(specs, pbs, methods):
        plan = pb.plan.replace(trunc_frac=0.0, grid_method=m, grid_tile=64)
        planes = o.mean_w_planes(d["uvw"][:, 2].astype(np.float64), d["P"])
        wk = wp.make_wkernels(plan, pb.taper, planes, supports=[min(5, d["max_support"])] * d["P"])
        ws = wp.workspace(wp.grid_workspace_bytes(plan, wk.P, pb.vis.numel()), dev)
        G = torch.zeros((plan.image_size, plan.image_size), dtype=torch.complex64, device=dev)
        jobs.append(api.GridJob(plan, wk, pb.uvw, pb.vis, None, G, ws,
                                torch.zeros(2, dtype=torch.float64, device=dev)))
        refs.append(wp.grid(plan, wk, pb.uvw, pb.vis)[0].cpu().numpy())
    bws = api.grid_batch_workspace(dev)
    assert api.grid_batch_selftest(jobs, bws) == -6
    for j in jobs:
        assert float(torch.abs(j.grid).max()) == 0.0
    for fused in (True, False):   # the same context grids correctly afterwards, in both forms
        for j in jobs:
            j.grid.zero_()
        api.grid_batch(jobs, bws, fused=fused)
        torch.cuda.synchronize()
        assert api.grid_batch_status(bws) == 0
        for j, r in zip(jobs, refs):
            assert np.abs(j.grid.cpu().numpy() - r).max() <= 1e-5 * np.abs(r).max()
