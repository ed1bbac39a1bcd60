"""Many independent imaging problems of uneven size in one CUDA-graph launch.

Each problem (its own grid size, plane count, visibilities) runs the whole path --
Hankel kernel generation, gridding, dirty image -- through the C ABI.  After a set-up
pass (plane values, transform matrices, supports by 1 % truncation read back once so that
each cache is laid out compactly, cuFFT plans, autotuned launch shapes) the steady-state
step of every problem is captured into one CUDA graph: the problems are spread over a few
side streams (largest first, round robin) forked from and joined back into the capture
stream, so small problems overlap with large ones and the host issues one launch for the
whole batch.  `run_sequential` runs the same steps one problem at a time for comparison.
With persistent=True the gridding of all problems instead runs in persistent launches that pull
(problem, plane, tile) work from one device queue per gridder kind (``api.grid_batch``).
"""
from __future__ import annotations

import dataclasses

import torch

from . import api
from .api import Plan, WKernels
from .autotune import GRID_CHOICES, KERNELGEN_CHOICES, Autotuner


@dataclasses.dataclass
class Problem:
    plan: Plan                 # geometry; trunc_frac > 0 selects the 1 % truncation supports
    taper: torch.Tensor        # [R] float32
    uvw: torch.Tensor          # [3V] float32
    vis: torch.Tensor          # [V] complex64
    P: int                     # number of |w| planes
    weight: torch.Tensor | None = None   # [V] float32 visibility weights (None: all 1)


class _State:
    def __init__(self, pb: Problem, tuner: Autotuner | None):
        dev = pb.vis.device
        self.pb = pb
        self.V = pb.vis.numel()
        self.w_planes = api.plane_values(pb.uvw, pb.P)
        plan = pb.plan
        ws = api.workspace(api.kernelgen_workspace_bytes(plan.replace(kernelgen="tf32x3"), pb.P), dev)
        api.kernelgen_prepare(plan, pb.P, ws)
        _, _, sup = api.hankel_radial(plan, pb.taper, self.w_planes, ws)
        sup_host = sup.cpu().tolist() if sup is not None else [plan.max_support] * pb.P
        self.plan = plan.replace(trunc_frac=0.0)
        self.support = torch.tensor(sup_host, dtype=torch.int32, device=dev)
        off_host = api.kernel_layout(self.plan, sup_host)
        self.offsets = torch.tensor(off_host, dtype=torch.int64, device=dev)
        self.ws = ws
        self.radial = torch.empty((pb.P, plan.geometry().k_out), dtype=torch.complex64, device=dev)
        self.spline_m = torch.empty_like(self.radial)
        self.cache = torch.empty(off_host[-1], dtype=torch.complex64, device=dev)
        self.grid_ws = api.workspace(max(api.grid_workspace_bytes(self.plan.replace(grid_method=m, grid_tile=t),
                                                                  pb.P, self.V)
                                         for m, t in list(GRID_CHOICES) + [(3, 64)]), dev)
        N = plan.image_size
        self.grid = torch.zeros((N, N), dtype=torch.complex64, device=dev)
        self.image = torch.empty((N, N), dtype=torch.float32, device=dev)
        self.stats = torch.zeros(2, dtype=torch.float64, device=dev)
        self.wk = WKernels(self.w_planes, self.support, self.offsets, self.cache, self.radial, self.spline_m)
        if tuner is not None:
            self._tune(tuner)

    def _tune(self, tuner: Autotuner) -> None:
        pb = self.pb
        k1 = Autotuner.key("kernelgen", pb.plan.image_size, pb.P, pb.plan.max_support)

        def run_kg(kg):
            self.kernels(self.plan.replace(kernelgen=kg))

        kg = tuner.choose(k1, list(KERNELGEN_CHOICES), run_kg)
        self.plan = self.plan.replace(kernelgen=kg)
        self.kernels(self.plan)
        k2 = Autotuner.key("grid", pb.plan.image_size, pb.P, pb.plan.max_support, self.V)

        def run_grid(mt):
            api.grid(self.plan.replace(grid_method=int(mt[0]), grid_tile=int(mt[1])), self.wk, pb.uvw, pb.vis,
                     pb.weight, self.grid, self.grid_ws, self.stats)

        m, t = tuner.choose(k2, [list(c) for c in GRID_CHOICES], run_grid)
        self.plan = self.plan.replace(grid_method=int(m), grid_tile=int(t))

    def kernels(self, plan: Plan) -> None:
        api.hankel_radial(plan, self.pb.taper, self.w_planes, self.ws, self.radial, self.spline_m)
        api.resample(plan, self.radial, self.spline_m, self.support, self.offsets, self.cache)

    def step(self) -> None:
        """Kernel generation + gridding + dirty image of this problem on the current stream."""
        self.kernels(self.plan)
        self.grid.zero_()
        self.stats.zero_()
        api.grid(self.plan, self.wk, self.pb.uvw, self.pb.vis, self.pb.weight, self.grid, self.grid_ws, self.stats)
        # normalised by the weights actually gridded (drops and weights included), read on the device
        api.dirty_image(self.plan, self.pb.taper, self.grid, self.stats, self.image)

    def cost(self) -> float:
        taps = float(self.V) * float((2 * self.pb.plan.max_support + 1) ** 2) / 4.0
        return taps + 64.0 * float(self.offsets[-1].item())


class BatchImager:
    """persistent=False: each problem's whole step (its own tuned gridder) on one of a few forked
    streams.  persistent=True: kernel generation of every problem on the forked streams, then
    the gridding of ALL problems in persistent launches pulling work from one device queue per
    gridder kind (``api.grid_batch``: the record orderings of every problem, then slot items for problems tuned to the slot gridder, row-owned tiles of 64
    cells for the rest, largest problems first), then the images."""

    def __init__(self, problems: list[Problem], n_streams: int = 4, tuner: Autotuner | None = None,
                 persistent: bool = False):
        self.states = [_State(pb, tuner) for pb in problems]
        self.n_streams = max(1, n_streams)
        self.persistent = persistent
        self.graph: torch.cuda.CUDAGraph | None = None
        dev = problems[0].vis.device
        self.bws = api.grid_batch_workspace(dev)
        order = sorted(range(len(self.states)), key=lambda i: -self.states[i].cost())
        # each problem's tuned gridder when it is the slot method (9), else the row-owned tiles (3)
        self.jobs = [api.GridJob(self.states[i].plan.replace(
                                     grid_method=9 if self.states[i].plan.grid_method == 9 else 3, grid_tile=64),
                                 self.states[i].wk,
                                 self.states[i].pb.uvw, self.states[i].pb.vis, self.states[i].pb.weight,
                                 self.states[i].grid, self.states[i].grid_ws, self.states[i].stats)
                     for i in order]
        self.run_sequential()          # plans, tuning and code loading outside any capture
        if persistent:
            self._persistent_step(torch.cuda.current_stream(), [torch.cuda.current_stream()],
                                  [list(range(len(self.states)))])
        torch.cuda.synchronize()

    @property
    def images(self) -> list[torch.Tensor]:
        return [s.image for s in self.states]

    def total_visibilities(self) -> int:
        return sum(s.V for s in self.states)

    def dropped(self) -> float:
        return float(sum(float(s.stats[1].item()) for s in self.states))

    def run_sequential(self) -> None:
        for s in self.states:
            s.step()

    def _fork_join(self, cap: torch.cuda.Stream, streams, lanes) -> None:
        fork = torch.cuda.Event()
        fork.record(cap)
        joins = []
        for st, lane in zip(streams, lanes):
            st.wait_event(fork)
            with torch.cuda.stream(st):
                for i in lane:
                    self.states[i].step()
                ev = torch.cuda.Event()
                ev.record(st)
            joins.append(ev)
        for ev in joins:
            cap.wait_event(ev)

    def _persistent_step(self, cap: torch.cuda.Stream, streams, lanes) -> None:
        fork = torch.cuda.Event()
        fork.record(cap)
        joins = []
        for st, lane in zip(streams, lanes):
            st.wait_event(fork)
            with torch.cuda.stream(st):
                for i in lane:
                    self.states[i].kernels(self.states[i].plan)
                ev = torch.cuda.Event()
                ev.record(st)
            joins.append(ev)
        for ev in joins:
            cap.wait_event(ev)
        with torch.cuda.stream(cap):
            for s in self.states:
                s.grid.zero_()
                s.stats.zero_()
            api.grid_batch(self.jobs, self.bws)
            for s in self.states:
                api.dirty_image(s.plan, s.pb.taper, s.grid, s.stats, s.image)

    def status(self) -> int:
        """Device status of the last persistent gridding launch (0 or WP_ERR_TIMEOUT)."""
        return api.grid_batch_status(self.bws)

    def capture(self) -> None:
        order = sorted(range(len(self.states)), key=lambda i: -self.states[i].cost())
        lanes = [[] for _ in range(self.n_streams)]
        for j, i in enumerate(order):
            lanes[j % self.n_streams].append(i)
        streams = [torch.cuda.Stream() for _ in range(self.n_streams)]
        cap = torch.cuda.Stream()
        # one uncaptured pass on the same streams first: the library keeps one cuFFT plan per
        # stream (concurrent branches never share a work area), and a plan cannot be created
        # inside a capture
        step = self._persistent_step if self.persistent else self._fork_join
        torch.cuda.synchronize()
        step(cap, streams, lanes)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            step(cap, streams, lanes)
        self.graph = g

    def replay(self) -> None:
        if self.graph is None:
            self.capture()
        self.graph.replay()
