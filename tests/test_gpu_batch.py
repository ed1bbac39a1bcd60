"""Batched uneven imaging problems: the graph-replayed batch gives the same dirty images as
running the problems one at a time and as the plain API calls; the autotuner's choices do
not change results."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problems(dev):
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.batch import Problem

    specs = synth.batch_problems(n=5, seed=7, sizes=(256, 512), planes=(8, 40), vis=(2000, 60000))
    out = []
    for d in specs:
        R = 256
        plan = wp.Plan(d["N"], d["cell_size"], 8, d["max_support"], 3, 0.01, R, "cubic", "fp32")
        taper = torch.tensor(synth.gaussian_taper_samples(d["N"], d["cell_size"], R), dtype=torch.float32,
                             device=dev)
        uvw = torch.tensor(d["uvw"], device=dev).reshape(-1)
        vis = torch.tensor(synth.predict(d["uvw"], d["sky"]), device=dev)
        out.append(Problem(plan, taper, uvw, vis, d["P"]))
    return out


def test_graph_batch_matches_sequential_and_direct_calls(tmp_path):
    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.autotune import Autotuner
    from paper_1904_08463_gb300.batch import BatchImager

    dev = torch.device("cuda")
    pbs = _problems(dev)
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
