"""Autotuner for the tunable launch shapes of the imaging path.

Three choices do not change results beyond the kernel tolerance, only speed: the
kernel-generation route of the Hankel transform (FP32 SIMT, or the tcgen05 matrix product with
TF32x3, BF16x3 or BF16x6 split operands -- all within 1e-6 of the FP64 oracle on the caches),
and the gridder's method (register tile; shared-memory tiles with the footprint spread over
the lanes, per-warp copies, or warp-owned rows; warp-owned rows with taps interpolated from
the radial line) and tile side (32 or 64 cells).  For a problem class -- grid size, plane
count, maximum support, visibility count, each bucketed -- the tuner times every
candidate on the problem itself with CUDA events and keeps the fastest; the table can be
saved as JSON and reloaded so that a tuned class is never timed again.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable

import torch

KERNELGEN_CHOICES = ("fp32", "tf32x3", "bf16x3", "bf16x6")
TILE_CHOICES = (32, 64)
GRID_CHOICES = tuple((m, t) for m in (0, 1, 3, 4, 5, 6, 7, 8) for t in TILE_CHOICES) + ((2, 32), (9, 64))   # (grid_method, grid_tile)


def _bucket(x: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))


class Autotuner:
    def __init__(self, path: str | None = None):
        self.path = path
        self.table: dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as fh:
                self.table = json.load(fh)

    @staticmethod
    def key(kind: str, N: int, P: int, s_max: int, V: int = 0) -> str:
        return f"{kind}:N{N}:P{_bucket(P)}:S{s_max}:V{_bucket(V) if V else 0}"

    def save(self) -> None:
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(self.table, fh, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def choose(self, key: str, candidates, run: Callable[[object], None], reps: int = 3):
        """Return the fastest candidate for `key` (timing each with CUDA events if the key is
        new).  `run(candidate)` must enqueue one complete execution on the current stream."""
        if key in self.table:
            return self.table[key]["best"]
        times = {}
        for c in candidates:
            run(c)                                   # warm-up (plans, code loading)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                run(c)
            b.record()
            torch.cuda.synchronize()
            times[json.dumps(c)] = a.elapsed_time(b) / reps
        best = min(times, key=times.get)
        self.table[key] = {"best": json.loads(best), "ms": times}
        self.save()
        return self.table[key]["best"]
