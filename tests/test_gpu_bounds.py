"""The checked build (-DWP_CHECK_BOUNDS): the library compiled with index checks on the tap reads
and grid-cell accesses of the gridders (grid_method 3 and 9, per call and in the persistent
batch), the degridders (0 and 9) and the kernel-cache rows the resample writes.  On the
benchmark's geometries -- a seeded 65,536-visibility subset of the full-imaging workload with
BF16x3 kernels, 1 % supports chosen on the device and the maximum-support cache layout, and a
few small uneven problems in one persistent batch -- no access may fall outside its buffer
(wp_bounds_status reads 0), and the checked build's grids and visibilities equal the default
build's.

The checked library runs in a child process (the package loads one library per process)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_1904_08463_gb300._lib as L
if sys.argv[2] != "-":
    L.LIB_PATH = sys.argv[2]
import torch
import paper_1904_08463_gb300 as wp
from paper_1904_08463_gb300 import api
from paper_1904_08463_gb300.imager import Imager
import synth

lib = L.load()
dev = torch.device("cuda")
out = {}


def status():
    v = ctypes.c_uint64()
    rc = lib.wp_bounds_status(ctypes.byref(v), 1)
    return [int(rc), int(v.value)]


d = synth.full_imaging()
rng = np.random.default_rng(5)
idx = np.sort(rng.choice(d["uvw"].shape[0], 65536, replace=False))
uvw = np.ascontiguousarray(d["uvw"][idx])
vis = synth.predict(uvw, d["sky"]).astype(np.complex64)
N, dl, R, P = d["N"], d["cell_size"], 512, 512
plan = wp.Plan(N, dl, 8, 127, 3, 0.01, R, "cubic", "bf16x3")
tap = torch.tensor(synth.gaussian_taper_samples(N, dl, R), dtype=torch.float32, device=dev)
u = torch.tensor(uvw, device=dev).reshape(-1)
v = torch.tensor(vis, device=dev)
im = Imager(plan, tap, u, P)
im.kernels()
torch.cuda.synchronize()
out["resample"] = status()
sums = {}
for m in (3, 9):
    G, st = wp.grid(im.plan.replace(grid_method=m, grid_tile=64), im.wk, u, v)
    torch.cuda.synchronize()
    out[f"grid{m}"] = status()
    sums[f"grid{m}"] = [float(G.real.double().sum()), float(G.imag.double().sum()), float(G.abs().max())]
    if m == 9:
        Gm = G
for m in (0, 9):
    vo = wp.degrid(im.plan.replace(grid_method=m, grid_tile=64), im.wk, u, Gm)
    torch.cuda.synchronize()
    out[f"degrid{m}"] = status()
    sums[f"degrid{m}"] = [float(vo.real.double().sum()), float(vo.imag.double().sum())]

# persistent batch: small uneven problems, row-owned and slot jobs in one launch
jobs = []
for i, (n_side, P_i, V_i, m) in enumerate([(512, 24, 3000, 3), (1024, 40, 9000, 9), (512, 16, 5000, 9)]):
    dl_i = float(np.deg2rad(8.0) / n_side)
    uvw_i = synth.track_uvw(n_dumps=-(-V_i // 2016), seed=70 + i, max_vis=V_i)
    uvw_i, _ = synth.scale_to_grid(uvw_i, (n_side / 2 - 12) * (1.0 / (n_side * dl_i)))
    p_i = wp.Plan(n_side, dl_i, 8, 9, 3, 0.0, 256, "cubic", "tf32x3", grid_method=m, grid_tile=64)
    tap_i = torch.tensor(synth.gaussian_taper_samples(n_side, dl_i, 256), dtype=torch.float32, device=dev)
    u_i = torch.tensor(uvw_i, device=dev).reshape(-1)
    planes = np.linspace(0.0, float(np.abs(uvw_i[:, 2]).max()) + 1.0, P_i)
    wk = wp.make_wkernels(p_i, tap_i, planes, supports=[9] * P_i)
    v_i = torch.ones(uvw_i.shape[0], dtype=torch.complex64, device=dev)
    ws = wp.workspace(wp.grid_workspace_bytes(p_i, P_i, v_i.numel()), dev)
    G = torch.zeros((n_side, n_side), dtype=torch.complex64, device=dev)
    jobs.append(api.GridJob(p_i, wk, u_i, v_i, None, G, ws, torch.zeros(2, dtype=torch.float64, device=dev)))
bws = api.grid_batch_workspace(dev)
api.grid_batch(jobs, bws)
torch.cuda.synchronize()
out["batch_status"] = api.grid_batch_status(bws)
out["batch"] = status()
sums["batch"] = [float(j.grid.abs().sum()) for j in jobs]
out["sums"] = sums
print(json.dumps(out))
"""


def _run(lib_path: str) -> dict:
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, lib_path], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_finds_no_access_outside_its_buffer():
    from paper_1904_08463_gb300 import build

    checked = _run(build.build_checked())
    for k in ("resample", "grid3", "grid9", "degrid0", "degrid9", "batch"):
        rc, first = checked[k]
        assert rc == 0, (k, rc)
        assert first == 0, f"{k}: first access outside its buffer: site {first >> 48}, index {first & (2**48 - 1)}"
    assert checked["batch_status"] == 0
    # the checks change no result: the default build gives the same sums
    plain = _run("-")
    assert plain["resample"][0] == -8          # the default build keeps no checks
    for k, a in checked["sums"].items():
        b = plain["sums"][k]
        for x, y in zip(a, b):
            assert abs(x - y) <= 1e-5 * max(abs(y), 1e-30) + 1e-6, (k, a, b)
