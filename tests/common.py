"""Shared helpers for the GPU parity tests (input shapes and comparisons only)."""
from __future__ import annotations

import numpy as np

import synth

KERNEL_TOL = 1e-5        # relative L2 per kernel (radial line and cache), vs the FP64 oracle
IMAGE_TOL = 1e-4         # max |dirty image error| / max |oracle image| inside the circle


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb else float(np.linalg.norm(a))


def f32(x):
    """Round an input array to float32 (what the CUDA path receives) and return float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def supports_match(gpu_sup, oracle_radial, oracle_sup, tau, os_, rel=1e-4) -> bool:
    """Supports must agree exactly unless the oracle's radial line sits within `rel` of the
    truncation threshold at the radii that decide them (an FP32 vs FP64 near-tie)."""
    gpu_sup = np.asarray(gpu_sup)
    oracle_sup = np.asarray(oracle_sup)
    for p in np.flatnonzero(gpu_sup != oracle_sup):
        a = np.abs(oracle_radial[p])
        thr = tau * a.max()
        lo, hi = sorted((int(gpu_sup[p]), int(oracle_sup[p])))
        ks = np.arange((lo - 1) * os_ + 1, hi * os_ + 1)
        ks = ks[(ks >= 0) & (ks < a.size)]
        if not np.any(np.abs(a[ks] - thr) <= rel * thr):
            return False
    return True

