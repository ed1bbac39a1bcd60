"""Benchmark: Hankel w-kernel generation (w-kernels/s) and gridding (Mvis/s) on one GB300.

Headline workload (kernel-generation batch): 1024 signed w-planes linearly spaced in
[-20000, 20000] wavelengths (512 distinct |w| kernels, Section 4.1), radial profile
length 4096, oversampling 8, support growing with |w| from 7 to 127, 8 degree FOV on a
4096^2 grid, Gaussian anti-aliasing taper.  One step = screen + Hankel transform (batched
matrix product) + spline + resampling of all 512 planes into the oversampled cache
(6.05 GB written per step, far larger than L2, so no flush is needed between steps).

Also measured in the same run (reported under "imaging"): full imaging with 8M
visibilities (64-antenna 8 h track at dec -30, 1.4 GHz), 512 |w|-planes, 1 % truncation,
S_max 127, 4096^2 grid: kernel generation + gridding + dirty image per step, with the FP64
oracle's gridding rate on a seeded 65,536-visibility subset beside it.  Under "batched": 48
independent problems of uneven size as one CUDA graph, one at a time, and through the
persistent batch gridder.  Under "differentiation": forward prediction + hand-written backward
of a chi-squared loss to a 4096^2 model image and the radial taper, 2M visibilities.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

# DRAM read + write bytes of one k_resample launch on the 512-plane batch, from an ncu capture
# of the every-2nd-plane case scaled by the ratio of algorithmic bytes.  Reported only while the
# resample's source (its section of kernelgen.cu and the shared tap evaluation) is the one it
# was measured on.
RESAMPLE_TRAFFIC = {"bytes_per_launch": 5.9288e+09, "source_sha1": "34ed20659d55"}

GRID_METHOD_NAMES = {0: "register tile", 1: "shared-memory tile, footprint over the lanes (atomics)",
                     2: "warp-private shared-memory tiles", 3: "shared-memory tile, rows owned by warps",
                     4: "rows owned by warps, taps interpolated from the radial line",
                     5: "shared-memory tile over groups of 8 planes", 6: "row registers over groups of 8 planes",
                     7: "rows owned by warps, 2 visibilities per update", 8: "rows owned by warps, 4 visibilities per update",
                     9: "slots: register sums along a Morton curve (Romein's work distribution)"}

METRIC = "w-kernels/s (Hankel vs 2D-FFT) and Mvis/s gridded, 1 GB300, at stated FP64 error"
N_IMG, FOV_DEG, R_KG, OS = 4096, 8.0, 4096, 8


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


def measure_compute_peaks(dev) -> dict:
    """FP32 FMA and TF32 tensor rates measured on this GPU in this run (the HBM and BF16 peaks
    come from MEASURED_PEAKS.json): FP32 = register-resident FMA chains (wp_probe_fp32_fma,
    8 blocks of 256 threads per SM), TF32 = torch.matmul of 8192^2 float32 matrices with TF32
    allowed (cuBLAS, 2 n^3 flops); each the best of 5 CUDA-event timings after a warm-up."""
    import ctypes

    import torch

    from paper_1904_08463_gb300 import _lib

    lib = _lib.load()
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    flops = ctypes.c_double()

    def fma():
        _lib.check("wp_probe_fp32_fma", lib.wp_probe_fp32_fma(4096, 8, ctypes.c_void_p(sink.data_ptr()),
                                                               ctypes.byref(flops), ctypes.c_void_p(st.cuda_stream)))

    def best(fn, n=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    ms_fma = best(fma)                       # the call fills `flops`
    fp32 = flops.value / (ms_fma * 1e-3) / 1e12
    # L2 rate of the gridder's tap-load shape: ten rows of 32 complex64 at random 8-byte offsets of
    # a 64 MB buffer (L2-resident), rows 67 values apart; best over 3, 4 and 8 blocks per SM
    tbuf = torch.zeros(8 << 20, dtype=torch.complex64, device=dev)
    nbytes = ctypes.c_double()
    l2 = 0.0
    for bps in (3, 4, 8):
        def taps():
            _lib.check("wp_probe_l2_taps", lib.wp_probe_l2_taps(
                ctypes.c_void_p(tbuf.data_ptr()), tbuf.numel(), 67, 2000, bps, ctypes.c_void_p(sink.data_ptr()),
                ctypes.byref(nbytes), ctypes.c_void_p(st.cuda_stream)))
        ms = best(taps)
        l2 = max(l2, nbytes.value / (ms * 1e-3) / 1e9)
    del tbuf
    n = 8192
    x = torch.randn(n, n, device=dev, dtype=torch.float32)
    y = torch.randn(n, n, device=dev, dtype=torch.float32)
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        tf32 = 2.0 * n ** 3 / (best(lambda: torch.matmul(x, y)) * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    del x, y
    hbm, bf16, src = _peaks()
    return {"fp32_fma_tflops": fp32, "tf32_tflops": tf32, "bf16_tflops": bf16, "hbm_gbs": hbm,
            "l2_tap_gbs": l2,
            "how": "FP32: FMA chains in registers, all SMs (wp_probe_fp32_fma); TF32: cuBLAS 8192^3 "
                   "torch.matmul with TF32 allowed; L2 taps: the gridder's tap-load shape on an "
                   "L2-resident 64 MB buffer (wp_probe_l2_taps); best of 5 CUDA-event timings; HBM and "
                   f"BF16: {src} MEASURED_PEAKS.json"}


def max_over_ranks(ms: float, device, world: int) -> float:
    """Replicas only (every rank runs the whole workload on its own GPU): the job's time is the
    slowest rank's, so value = ranks x work / max time."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def resample_source_hash():
    """sha1 of the resample kernel's source: its section of kernelgen.cu and the shared tap
    evaluation it inlines."""
    import hashlib

    base = os.path.join(ROOT, "paper_1904_08463_gb300", "csrc")
    try:
        kg = open(os.path.join(base, "kernelgen.cu"), "rb").read()
        hd = open(os.path.join(base, "wp_internal.cuh"), "rb").read()
    except OSError:
        return None
    a, b = kg.find(b"// K7: resample"), kg.find(b"}  // namespace wp")
    c = hd.find(b"__device__ __forceinline__ int skew(int k)")
    d = hd.find(b"#endif", c)
    if min(a, b, c, d) < 0:
        return None
    return hashlib.sha1(kg[a:b] + hd[c:d]).hexdigest()[:12]


def resample_traffic():
    h = resample_source_hash()
    return RESAMPLE_TRAFFIC["bytes_per_launch"] if h == RESAMPLE_TRAFFIC["source_sha1"] else None


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- workloads
def kernel_batch():
    dl = np.deg2rad(FOV_DEG) / N_IMG
    w_signed, aw, sup = synth.kernel_batch_planes()
    taper = synth.gaussian_taper_samples(N_IMG, dl, R_KG)
    return dict(N=N_IMG, cell_size=dl, w_signed=w_signed, w_abs=aw, support=sup, taper=taper)


def cache_bytes(sup) -> int:
    return int(sum(OS * OS * (2 * int(s) + 1) ** 2 * 8 for s in sup))


# --------------------------------------------------------------------------- oracle (CPU)
def oracle_kernel_rate(n_planes: int = 512):
    """The FP64 oracle as it stands, on n_planes planes spread evenly over the batch's |w|
    (all 512 by default: about 10-15 s on the host cores).  Per plane: screen, transform,
    spline and resample; the transform matrix, built once per geometry like the GPU's
    prepare step, is excluded.  Returns (w-kernels/s, extrapolated to the batch's support
    mix by tap count when sampled, threads, sample description)."""
    from oracle import oracle as o

    kb = kernel_batch()
    g = o.Geometry(N_IMG, kb["cell_size"], OS, 127, 7, 0.0, R_KG)
    tap = kb["taper"].astype(np.float32).astype(np.float64)
    o.hankel_matrix(g.radial_samples, g.r_max, g.rho())       # build once (not timed)
    pick = np.linspace(0, len(kb["w_abs"]) - 1, n_planes).round().astype(int)
    taps_sample = 0
    t0 = time.perf_counter()
    for p in pick:
        C = o.radial_kernel(g, tap, float(kb["w_abs"][p]))
        o.resample(g, C, int(kb["support"][p]))
        taps_sample += (2 * int(kb["support"][p]) + 1) ** 2
    dt = time.perf_counter() - t0
    # per-plane time scales with its tap count: extrapolate to the batch's mix
    taps_batch = sum((2 * int(s) + 1) ** 2 for s in kb["support"])
    t_batch = dt * taps_batch / taps_sample
    rate = len(kb["w_abs"]) / t_batch
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return rate, threads, (f"{n_planes} of 512 |w| planes (supports {int(kb['support'][pick].min())}.."
                           f"{int(kb['support'][pick].max())}) in {dt:.1f} s, extrapolated by tap count; "
                           f"transform matrix excluded; OpenMP over planes' transform rows and sub-kernels")


def oracle_grid_rate(n_vis: int = 65536, seed: int = 12):
    """The FP64 oracle's gridding as it stands (binning decisions + gridding, one thread), on a
    seeded subset of n_vis visibilities of the full-imaging workload (8M-visibility track set,
    512 planes from the subset's |w|, 1 % truncation supports, S_max 127); its kernel cache is
    built first and not timed.  Returns (Mvis/s, sample description)."""
    from oracle import oracle as o

    d = synth.full_imaging()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(d["uvw"].shape[0], n_vis, replace=False))
    uvw = np.ascontiguousarray(d["uvw"][idx])
    vis = synth.predict(uvw, d["sky"]).astype(np.complex64)
    N, dl, R = d["N"], d["cell_size"], 512
    g = o.Geometry(N, dl, OS, 127, 3, 0.01, R)
    tap = synth.gaussian_taper_samples(N, dl, R).astype(np.float32).astype(np.float64)
    planes = o.mean_w_planes(uvw[:, 2].astype(np.float64), 512)
    ks = o.wkernels(g, tap, planes)
    t0 = time.perf_counter()
    b = o.bin_vis(g, uvw, planes, ks.support)
    o.grid(g, ks, b, vis)
    dt = time.perf_counter() - t0
    taps = float(np.sum((2 * ks.support[b.plane[b.drop == 0]].astype(np.float64) + 1) ** 2))
    return n_vis / dt / 1e6, (f"{n_vis} seeded visibilities of the 8M full-imaging workload ({taps / n_vis:.0f} "
                              f"taps each), binning + gridding in {dt:.1f} s on one thread; kernel cache built "
                              "beforehand, not timed")


def oracle_rate_one_thread(n_planes: int = 64):
    """The same oracle timing with one OpenMP thread (a child process: the thread count of
    the loaded oracle library is fixed), on n_planes planes spread over the batch."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = ("import json, bench; r, t, s = bench.oracle_kernel_rate(%d); print(json.dumps(r))" % n_planes)
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                             timeout=300)
        return float(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


# ------------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300 import _lib

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    kb = kernel_batch()
    if args.plane_stride > 1:
        for key in ("w_abs", "support"):
            kb[key] = kb[key][::args.plane_stride]
        kb["w_signed"] = kb["w_signed"][::args.plane_stride]
    P = len(kb["w_abs"])
    plan = wp.Plan(N_IMG, kb["cell_size"], OS, 127, 7, 0.0, R_KG, "cubic", args.kernelgen)
    g = plan.geometry()
    taper_d = torch.tensor(kb["taper"], dtype=torch.float32, device=dev)
    wpl_d = torch.tensor(kb["w_abs"], dtype=torch.float64, device=dev)
    sup_host = [int(s) for s in kb["support"]]
    sup_d = torch.tensor(sup_host, dtype=torch.int32, device=dev)
    off_host = wp.kernel_layout(plan, sup_host)
    off_d = torch.tensor(off_host, dtype=torch.int64, device=dev)
    ws = wp.workspace(wp.kernelgen_workspace_bytes(plan, P), dev)
    wp.kernelgen_prepare(plan, P, ws)
    radial = torch.empty((P, g.k_out), dtype=torch.complex64, device=dev)
    spline_m = torch.empty_like(radial)
    cache = torch.empty(1 if args.hankel_only else off_host[-1], dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()
    lib = _lib.load()
    cplan = plan.c()
    import ctypes

    def step(ev=None):
        _lib.check("wp_hankel_radial", lib.wp_hankel_radial(
            ctypes.byref(cplan), ctypes.c_void_p(taper_d.data_ptr()), ctypes.c_void_p(wpl_d.data_ptr()), P,
            ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(radial.data_ptr()),
            ctypes.c_void_p(spline_m.data_ptr()), None, ctypes.c_void_p(stream.cuda_stream)))
        if ev is not None:
            ev[0].record(stream)
        if args.hankel_only:
            if ev is not None:
                ev[1].record(stream)
            return
        _lib.check("wp_resample", lib.wp_resample(
            ctypes.byref(cplan), ctypes.c_void_p(radial.data_ptr()), ctypes.c_void_p(spline_m.data_ptr()), P,
            ctypes.c_void_p(sup_d.data_ptr()), ctypes.c_void_p(off_d.data_ptr()),
            ctypes.c_void_p(cache.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream)))
        if ev is not None:
            ev[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    # keep the same load on for about a second so that the clock sampler sees it
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 1.0:
        for _ in range(20):
            step()
        torch.cuda.synchronize()
    clk = clocks.stop()
    clk["note"] = "sampled every 200 ms over the timed steps plus ~1 s of the same steps right after"
    # context for the write-only resample: the same GPU writing the cache's bytes with a plain
    # fill (library kernel, outside the step; the next step rewrites the cache)
    write_gbs = None
    if not args.hankel_only:
        fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cache.zero_()
        fa.record(stream)
        for _ in range(5):
            cache.zero_()
        fb.record(stream)
        torch.cuda.synchronize()
        write_gbs = cache.numel() * 8 * 5 / (fa.elapsed_time(fb) * 1e-3) / 1e9
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), dev, world)
    ms_step = ms_total / args.steps
    resample_ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    value = world * P / (ms_step * 1e-3)
    bytes_cache = cache_bytes(sup_host)
    # algorithmic bytes of one resample launch: cache written + each plane's radial line and
    # spline coefficients read once (re-reads of the line by the launch's other blocks are L2
    # traffic of this implementation, not algorithmic bytes)
    alg_bytes = bytes_cache + P * 16 * min(g.k_out, OS * 127 + 2)
    hbm, bf16, src = _peaks()
    achieved = alg_bytes / (resample_ms * 1e-3) / 1e9

    # ---- end to end through the C ABI with host buffers -----------------------------
    e2e = None
    if args.e2e:
        e2e = measure_e2e(args, world, P, kb, sup_host, off_host, cache, taper_d, wpl_d, sup_d, off_d, step, stream)
    out = build_line(args, world, P, kb, ms_step, resample_ms, bytes_cache, alg_bytes, hbm, src, achieved,
                     e2e, clk)
    if write_gbs is not None:
        out["roofline"]["write_stream"] = {
            "gbs": write_gbs, "frac": achieved / write_gbs,
            "note": "the same GPU filling the cache's bytes with a plain write stream (torch zero_), timed "
                    "right after the steps; a write-only kernel can exceed the copy bandwidth that 'peak' is"}
    if args.routes and not args.hankel_only:
        out["routes"] = time_routes(args, kb, plan, taper_d, wpl_d, sup_host, ws, radial, spline_m, cache,
                                    sup_d, off_d, ms_step)
    if rank == 0:
        out["measured_peaks"] = args.peaks = measure_compute_peaks(dev)
        if args.routes and not args.hankel_only and "routes" in out:
            add_tensor_fractions(out["routes"], plan, P, args.peaks)
    if args.imaging and rank == 0:
        out["imaging"] = run_imaging(args, dev)
    if args.batch and rank == 0:
        out["batched"] = run_batch(args, dev)
    if args.grad and rank == 0:
        out["differentiation"] = run_grad(args, dev)
    if rank == 0 and args.cpu_baseline:
        rate, thr, sample = oracle_kernel_rate()
        out["cpu_baseline"] = {"value": rate, "unit": "w-kernels/s", "cores": thr, "kind": "oracle",
                               "sample": sample}
        one = oracle_rate_one_thread()
        if one is not None:
            # the paper's parallel efficiency (Section 6): T_1 / (n T_n) = rate_n / (n rate_1)
            out["cpu_baseline"].update({"value_1_thread": one, "parallel_efficiency": rate / (thr * one)})
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def time_routes(args, kb, plan, taper_d, wpl_d, sup_host, ws, radial, spline_m, cache, sup_d, off_d,
                headline_ms):
    """The same batch through the other kernel-generation routes on the same GPU: the plain
    FP32 SIMT Hankel product and the standard 2D-FFT route (Alg. 1 with workspace
    undersampling, M = 256, 2048^2 transforms, circular support)."""
    import torch

    import paper_1904_08463_gb300 as wp

    P = len(kb["w_abs"])
    res = {args.kernelgen + "_hankel": {"ms_per_step": headline_ms, "w_kernels_per_s": P / (headline_ms * 1e-3)}}

    def timeit(fn, n):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    # the other matrix routes on the same prepared workspace (its layout and tables serve every
    # route): FP32 SIMT; TF32 hi/lo (3 products); BF16 hi/lo (3 products, kind::f16 at twice the
    # TF32 rate, ~2e-6 error); BF16 hi/lo/lo2 (6 products, TF32x3's accuracy)
    for kg in ("fp32", "tf32x3", "bf16x3", "bf16x6"):
        if kg == args.kernelgen:
            continue
        pk = plan.replace(kernelgen=kg)

        def route(pk=pk):
            wp.hankel_radial(pk, taper_d, wpl_d, ws, radial, spline_m)
            wp.resample(pk, radial, spline_m, sup_d, off_d, cache)

        ms = timeit(route, max(3, min(args.steps, 10)))
        res[kg + "_hankel"] = {"ms_per_step": ms, "w_kernels_per_s": P / (ms * 1e-3)}
    # the radial stage alone (screen, transform, truncation + spline) of every matrix route
    for kg in ("fp32", "tf32x3", "bf16x3", "bf16x6"):
        pk = plan.replace(kernelgen=kg)
        ms = timeit(lambda pk=pk: wp.hankel_radial(pk, taper_d, wpl_d, ws, radial, spline_m),
                    max(5, min(args.steps, 20)))
        res.setdefault(kg + "_hankel", {})["radial_stage_ms"] = ms
    # the projection-slice realisation of the Hankel transform (the variant the paper timed):
    # workspace image summed over one axis, zero-padded by os, batched 1D cuFFT
    p3 = plan.replace(kernelgen="projslice")
    ws3 = wp.workspace(wp.kernelgen_workspace_bytes(p3, P))
    wp.kernelgen_prepare(p3, P, ws3)

    def projslice():
        wp.hankel_radial(p3, taper_d, wpl_d, ws3, radial, spline_m)
        wp.resample(p3, radial, spline_m, sup_d, off_d, cache)

    ms = timeit(projslice, max(3, min(args.steps, 10)))
    res["projslice_hankel"] = {"ms_per_step": ms, "w_kernels_per_s": P / (ms * 1e-3),
                               "line": "M=256 workspace projected, 2048-point 1D cuFFT per plane"}
    del ws3
    fws = wp.workspace(int(wp._lib.load().wp_fft_workspace_bytes(__import__("ctypes").byref(plan.c()), P)))
    import ctypes

    lib = wp._lib.load()

    def fft_route():
        wp._lib.check("wp_fft_wkernels", lib.wp_fft_wkernels(
            ctypes.byref(plan.c()), ctypes.c_void_p(taper_d.data_ptr()), ctypes.c_void_p(wpl_d.data_ptr()), P,
            ctypes.c_void_p(sup_d.data_ptr()), ctypes.c_void_p(off_d.data_ptr()), 1,
            ctypes.c_void_p(fws.data_ptr()), fws.numel(), ctypes.c_void_p(cache.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    ms = timeit(fft_route, 2)
    res["fft2d"] = {"ms_per_step": ms, "w_kernels_per_s": P / (ms * 1e-3),
                    "workspace": "M=256 -> 2048^2 complex64 per plane, batched cuFFT C2C"}
    res["speedup_hankel_vs_fft2d"] = ms / headline_ms
    del fws
    return res


def add_tensor_fractions(routes, plan, P, peaks):
    """Fraction of the tensor peak of each tcgen05 route's transform: split products x
    2 K_out R_pad 2 P_pad flop over the radial stage's time (screen and spline included, so the
    fraction is a lower bound), against the measured TF32 (this run) or BF16 (MEASURED_PEAKS)
    rate."""
    g = plan.geometry()
    p_pad = (P + 63) // 64 * 64
    flop_one = 2.0 * g.k_out * g.r_pad * 2 * p_pad
    for kg, prods, peak_key in (("tf32x3", 3, "tf32_tflops"), ("bf16x3", 3, "bf16_tflops"),
                                ("bf16x6", 6, "bf16_tflops")):
        r = routes.get(kg + "_hankel")
        if not r or "radial_stage_ms" not in r or not peaks.get(peak_key):
            continue
        tf = prods * flop_one / (r["radial_stage_ms"] * 1e-3) / 1e12
        r["transform"] = {"products": prods, "gflop": prods * flop_one / 1e9, "tflops_over_radial_stage": tf,
                          "peak": peaks[peak_key], "peak_kind": peak_key, "frac_lower_bound": tf / peaks[peak_key]}


def measure_e2e(args, world, P, kb, sup_host, off_host, cache, taper_d, wpl_d, sup_d, off_d, step, stream):
    import torch

    pin_cache = torch.empty(off_host[-1], dtype=torch.complex64, pin_memory=True)
    h_taper = torch.tensor(kb["taper"], dtype=torch.float32).pin_memory()
    h_wpl = torch.tensor(kb["w_abs"], dtype=torch.float64).pin_memory()
    h_sup = torch.tensor(sup_host, dtype=torch.int32).pin_memory()
    h_off = torch.tensor(off_host, dtype=torch.int64).pin_memory()
    h2d = (h_taper.numel() * 4 + h_wpl.numel() * 8 + h_sup.numel() * 4 + h_off.numel() * 8)
    d2h = pin_cache.numel() * 8

    def e2e_step():
        taper_d.copy_(h_taper, non_blocking=True)
        wpl_d.copy_(h_wpl, non_blocking=True)
        sup_d.copy_(h_sup, non_blocking=True)
        off_d.copy_(h_off, non_blocking=True)
        step()
        pin_cache.copy_(cache, non_blocking=True)

    n_split = 4
    side = [torch.cuda.Stream() for _ in range(n_split)]
    bounds = [len(pin_cache) * i // n_split for i in range(n_split + 1)]

    def split_step():
        # same calls; the device-to-host read split over four streams (copy engines)
        taper_d.copy_(h_taper, non_blocking=True)
        wpl_d.copy_(h_wpl, non_blocking=True)
        sup_d.copy_(h_sup, non_blocking=True)
        off_d.copy_(h_off, non_blocking=True)
        step()
        done = torch.cuda.Event()
        done.record(stream)
        for i, st in enumerate(side):
            st.wait_event(done)
            with torch.cuda.stream(st):
                pin_cache[bounds[i]:bounds[i + 1]].copy_(cache[bounds[i]:bounds[i + 1]], non_blocking=True)
            back = torch.cuda.Event()
            back.record(st)
            stream.wait_event(back)

    n_e2e = max(2, min(args.steps, 5))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n_e2e

    # the same inputs in, but the kernels stay in HBM for the gridder and only a checksum of
    # the cache comes back (what a pipeline that grids on the same GPU reads)
    h_sum = torch.empty(2, dtype=torch.float32).pin_memory()

    def resident_step():
        taper_d.copy_(h_taper, non_blocking=True)
        wpl_d.copy_(h_wpl, non_blocking=True)
        sup_d.copy_(h_sup, non_blocking=True)
        off_d.copy_(h_off, non_blocking=True)
        step()
        h_sum.copy_(torch.view_as_real(cache[::4096]).sum(0), non_blocking=True)

    ms_copy = timed(e2e_step)
    ms_split = timed(split_step)
    ms_resident = timed(resident_step)
    e2e_ms = min(ms_copy, ms_split)
    return {"value": world * P / (e2e_ms * 1e-3), "unit": "w-kernels/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
            "method": ("device cache, read back to pinned host memory by "
                       + ("4 concurrent copies" if ms_split < ms_copy else "one copy")),
            "ms_one_copy": ms_copy, "ms_split_copies": ms_split,
            "kernels_resident": {"value": world * P / (ms_resident * 1e-3), "ms_per_step": ms_resident,
                                 "d2h_bytes_per_step": 8,
                                 "note": "same inputs copied in; the cache stays in HBM for gridding and "
                                         "only a two-float checksum of it is read back"}}


def build_line(args, world, P, kb, ms_step, resample_ms, bytes_cache, alg_bytes, hbm, src, achieved, e2e, clk):
    value = world * P / (ms_step * 1e-3)
    return {
        "metric": METRIC,
        "value": value,
        "unit": "w-kernels/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32x3": "tf32x3", "bf16x3": "bf16x3", "bf16x6": "bf16x6",
                  "projslice": "f32"}[args.kernelgen],
        "data": "synthetic",
        "config": {
            "workload": "kernel-generation batch: 1024 signed w-planes linspace[-20000,20000] "
                        "(512 distinct |w| kernels), R=4096, os=8, support 7..127 by |w|, "
                        "4096^2 grid, 8 deg FOV, Gaussian taper sigma=0.3 FOV",
            "kernelgen": args.kernelgen,
            "distinct_kernels_per_step": P,
            "delivered_kernels_per_step": int(len(kb["w_signed"])),
            "delivered_kernels_per_s": value * len(kb["w_signed"]) / P,
            "cache_bytes_per_step": bytes_cache,
            "l2": "no flush: each step writes a 6.05 GB cache (> 129 MB L2)",
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "roofline": {
            "kernel": "k_resample",
            "bound": "hbm",
            "achieved": achieved,
            "peak": hbm,
            "peak_source": f"{src} hbm_gbs (burst copy)",
            "unit": "GB/s",
            "frac": achieved / hbm,
            "traffic": resample_traffic(),
            "alg_bytes_per_launch": alg_bytes,
            "launch_ms": resample_ms,
            "share_of_step": resample_ms / ms_step,
        },
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
    }


def log(msg):
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def run_imaging(args, dev):
    """Full imaging: kernel generation (1 % truncation, max-support layout, no host sync)
    + gridding of 8M visibilities + dirty image, per step (the package's Imager step)."""
    import torch

    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.autotune import GRID_CHOICES, Autotuner
    from paper_1904_08463_gb300.imager import Imager

    log("imaging: generating inputs")
    d = synth.full_imaging(V=args.imaging_vis)
    N, dl = d["N"], d["cell_size"]
    uvw = torch.tensor(d["uvw"], device=dev)
    vis = synth.predict_torch(d["uvw"], d["sky"], dev)
    g = torch.Generator(device="cpu").manual_seed(d["noise_seed"])
    noise = torch.randn(vis.numel(), 2, generator=g, dtype=torch.float64) * d["noise_sigma"]
    vis = vis + torch.complex(noise[:, 0], noise[:, 1]).to(torch.complex64).to(dev)
    V = vis.numel()
    P = args.imaging_planes
    plan = wp.Plan(N, dl, OS, 127, 3, 0.01, 512, "cubic", args.kernelgen)
    taper = torch.tensor(synth.gaussian_taper_samples(N, dl, 512), dtype=torch.float32, device=dev)
    uvw_flat = uvw.reshape(-1)
    im = Imager(plan, taper, uvw_flat, P)        # plane values (Alg. 2 steps 1-3) on the GPU
    planes = im.w_planes.cpu().numpy()
    # the gridder's launch shape (method x tile) is picked by the autotuner on this problem
    tuner = Autotuner()
    choices = [list(c) for c in GRID_CHOICES]
    if args.grid_shape:
        choices = [[int(x) for x in args.grid_shape.split(",")]]
    im.autotune(uvw_flat, vis, None, tuner, choices)
    plan = im.plan
    img, stats, sup = im.image, im.stats, im.support

    def step(ev=None):
        im.kernels()
        if ev is not None:
            ev[0].record()
        im.grid_only(uvw_flat, vis)
        if ev is not None:
            ev[1].record()
        # normalised by the weight sum the gridder accumulated, read on the device (no sync)
        im.image_only()

    log("imaging: warm-up")
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    log("imaging: timed")
    n = max(1, min(args.steps, 3))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(n):
        step(evs[k])
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    grid_ms = float(np.mean([x.elapsed_time(y) for x, y in evs]))
    # end to end with host buffers: each step copies the visibilities (uvw, vis) in from
    # pinned host memory and reads the dirty image back
    uvw_h = uvw.reshape(-1).cpu().pin_memory()
    vis_h = vis.cpu().pin_memory()
    img_h = torch.empty(img.shape, dtype=img.dtype).pin_memory()

    def e2e_step():
        uvw_flat.copy_(uvw_h, non_blocking=True)
        vis.copy_(vis_h, non_blocking=True)
        step()
        img_h.copy_(img, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    a.record()
    for _ in range(n):
        e2e_step()
    b.record()
    torch.cuda.synchronize()
    ms_e2e = a.elapsed_time(b) / n
    sup_h = sup.cpu().numpy()
    # algorithmic work of gridding: 8 flop per tap of the (2S+1)^2 footprint of every
    # gridded visibility
    aw = np.abs(d["uvw"][:, 2].astype(np.float64))
    idx = np.clip(np.searchsorted(planes, aw), 1, P - 1)
    lower = np.where(np.abs(aw - planes[idx - 1]) <= np.abs(planes[idx] - aw), idx - 1, idx)
    taps = float(np.sum((2 * sup_h[lower].astype(np.float64) + 1) ** 2))
    flops = 8.0 * taps
    pk = getattr(args, "peaks", None) or {}
    fp32_peak = pk.get("fp32_fma_tflops") or 152 * 128 * 2 * 2.07e9 / 1e12
    fp32_src = ("measured in this run (register FMA chains on every SM)" if pk.get("fp32_fma_tflops")
                else "nominal: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz")
    st = stats.cpu().numpy()
    cpu = None
    if getattr(args, "cpu_baseline", False) and int(os.environ.get("RANK", "0")) == 0:
        log("imaging: CPU oracle on a subset")
        rate, sample = oracle_grid_rate()
        cpu = {"value": rate, "unit": "Mvis/s", "cores": 1, "kind": "oracle", "sample": sample}
    return {
        "cpu_baseline": cpu,
        "workload": f"full imaging: {V} visibilities (64-antenna 8 h track, dec -30, 1.4 GHz, uvw x "
                    f"{d['scale']:.3f}), 200 sources + 1 mJy noise, {P} |w|-planes (mean of "
                    f"equal-count chunks), 1% truncation, S_max 127, os 8, R 512, 4096^2 grid, 8 deg",
        "value": V / (ms * 1e-3) / 1e6,
        "unit": "Mvis/s",
        "ms_per_step": ms,
        "e2e": {"value": V / (ms_e2e * 1e-3) / 1e6, "unit": "Mvis/s", "ms_per_step": ms_e2e,
                "h2d_bytes_per_step": uvw_h.numel() * 4 + vis_h.numel() * 8,
                "d2h_bytes_per_step": img_h.numel() * 4},
        "grid_ms": grid_ms,
        "gridding_mvis_per_s": V / (grid_ms * 1e-3) / 1e6,
        "supports": {"min": int(sup_h.min()), "max": int(sup_h.max()), "mean": float(sup_h.mean())},
        "taps_per_vis": taps / V,
        "grid_launch_shape": {"method": GRID_METHOD_NAMES[plan.grid_method],
                              "tile": plan.grid_tile or 64, "chosen_by": "autotuner", "ms": tuner.table},
        "dropped": float(st[1]),
        "roofline": {"kernel": "k_grid", "bound": "alu", "achieved": flops / (grid_ms * 1e-3) / 1e12,
                     "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": flops / (grid_ms * 1e-3) / 1e12 / fp32_peak,
                     "peak_source": fp32_src,
                     "hbm_frac": (V * 24 + 2 * N * N * 8) / (grid_ms * 1e-3) / 1e9 / _peaks()[0],
                     # what bounds the cache gridders: every tap is one 8-byte L2 read
                     "l2": ({"achieved_gbs": 8.0 * taps / (grid_ms * 1e-3) / 1e9, "peak_gbs": pk["l2_tap_gbs"],
                             "frac": 8.0 * taps / (grid_ms * 1e-3) / 1e9 / pk["l2_tap_gbs"],
                             "peak_source": "measured in this run: the tap-load shape (ten rows of 32 "
                                            "complex64 at random offsets) on an L2-resident buffer"}
                            if pk.get("l2_tap_gbs") else None)},
    }


def run_batch(args, dev):
    """Independent imaging problems of uneven size (grid 512..4096, 32..512 planes, 1e5..4e6
    visibilities, per-problem seeds) in one CUDA-graph launch after autotuning, against the
    same steps issued one problem at a time."""
    import torch

    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.autotune import Autotuner
    from paper_1904_08463_gb300.batch import BatchImager, Problem

    log("batch: generating problems")
    specs = synth.batch_problems(n=args.batch_problems)
    pbs = []
    for d in specs:
        R = 512
        plan = wp.Plan(d["N"], d["cell_size"], OS, d["max_support"], 3, 0.01, R, "cubic", "tf32x3")
        taper = torch.tensor(synth.gaussian_taper_samples(d["N"], d["cell_size"], R), dtype=torch.float32,
                             device=dev)
        vis = synth.predict_torch(d["uvw"], d["sky"], dev)
        pbs.append(Problem(plan, taper, torch.tensor(d["uvw"], device=dev).reshape(-1), vis, d["P"]))
    log("batch: set-up and autotuning")
    tuner = Autotuner()
    b = BatchImager(pbs, n_streams=4, tuner=tuner)
    V = b.total_visibilities()

    def timeit(fn, n=3):
        fn()
        torch.cuda.synchronize()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        c.record()
        torch.cuda.synchronize()
        return a.elapsed_time(c) / n

    log("batch: timing")
    ms_seq = timeit(b.run_sequential)
    # the graph's fork width (side streams the problems are spread over) is tuned too
    by_streams = {}
    for ns in (2, 4, 8, 16):
        b.n_streams = ns
        b.graph = None
        b.capture()
        by_streams[ns] = timeit(b.replay)
    best_ns = min(by_streams, key=by_streams.get)
    ms_graph = by_streams[best_ns]
    # the same problems with their gridding in persistent launches (one device work queue over
    # every problem's record orderings, then its (plane, tile) or slot items), kernel generation and
    # images as before; captured in a graph
    b.persistent = True
    by_streams_p = {}
    for ns in (1, 2, 4):
        b.n_streams = ns
        b.graph = None
        b.capture()
        by_streams_p[ns] = timeit(b.replay)
    status = b.status()
    best_np = min(by_streams_p, key=by_streams_p.get)
    ms_pers = by_streams_p[best_np]
    choices = {}
    for k, v in tuner.table.items():
        choices[str(v["best"])] = choices.get(str(v["best"]), 0) + 1
    return {"workload": f"{len(pbs)} independent problems, grids {sorted(set(d['N'] for d in specs))}, "
                        f"planes {min(d['P'] for d in specs)}..{max(d['P'] for d in specs)}, "
                        f"{min(len(d['uvw']) for d in specs)}..{max(len(d['uvw']) for d in specs)} visibilities, "
                        "1% truncation, os 8, R 512",
            "visibilities": V, "ms_graph": ms_graph, "ms_sequential": ms_seq,
            "mvis_per_s_graph": V / (ms_graph * 1e-3) / 1e6, "mvis_per_s_sequential": V / (ms_seq * 1e-3) / 1e6,
            "speedup_graph_vs_sequential": ms_seq / ms_graph, "graph_streams": best_ns,
            "ms_graph_by_streams": by_streams,
            "ms_persistent": ms_pers, "mvis_per_s_persistent": V / (ms_pers * 1e-3) / 1e6,
            "speedup_persistent_vs_sequential": ms_seq / ms_pers, "persistent_kernelgen_streams": best_np,
            "ms_persistent_by_streams": by_streams_p, "persistent_status": status,
            "tuned_choices": choices, "dropped": b.dropped()}


def run_grad(args, dev):
    """Differentiation workload: the full-imaging geometry (4096^2, 512 planes) with 2M
    visibilities; one forward prediction from a 4096^2 float32 model image and a 512-sample
    taper, chi-squared loss, and the hand-written backward to both."""
    import torch

    import paper_1904_08463_gb300 as wp
    from paper_1904_08463_gb300.autograd import Predictor, chi2

    log("grad: inputs")
    d = synth.full_imaging(V=2 * 1024 * 1024)
    N, dl, R, P = d["N"], d["cell_size"], 512, 512
    uvw = torch.tensor(d["uvw"], device=dev).reshape(-1)
    vobs = synth.predict_torch(d["uvw"], d["sky"], dev)
    planes = wp.plane_values(uvw, P)
    # the backward pass grids with whichever gridder is faster on these inputs (timed below: the
    # slot walk, 9, the row-owned tile, 3, or the register tile, 0); the forward prediction
    # degrids with whichever degridder is faster (the warp per visibility, 0, or the slot walk in
    # reverse, 9)
    plan0 = wp.Plan(N, dl, OS, 127, 3, 0.01, R, "cubic", "tf32x3", 64, 9)
    taper0 = torch.tensor(synth.gaussian_taper_samples(N, dl, R), dtype=torch.float32, device=dev)
    ws = wp.kernelgen_prepare(plan0, P)
    _, _, sup = wp.hankel_radial(plan0, taper0, planes, ws)
    p_fix = plan0.replace(trunc_frac=0.0)
    V = vobs.numel()
    wk = wp.make_wkernels(p_fix, taper0, planes, supports=sup.cpu().tolist())
    X = torch.randn((N, N), dtype=torch.complex64, device=dev)
    dws = wp.workspace(max(wp.grid_workspace_bytes(p_fix.replace(grid_method=m), P, V) for m in (0, 3, 9)), dev)
    dout = torch.empty(V, dtype=torch.complex64, device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 3
    grid_ms_by = {}
    Gt = torch.zeros((N, N), dtype=torch.complex64, device=dev)
    for m in (9, 3, 0):
        pm = p_fix.replace(grid_method=m)
        for _ in range(2):
            wp.grid(pm, wk, uvw, vobs, None, Gt, dws)
        torch.cuda.synchronize()
        a.record()
        for _ in range(n):
            wp.grid(pm, wk, uvw, vobs, None, Gt, dws)
        b.record()
        torch.cuda.synchronize()
        grid_ms_by[m] = a.elapsed_time(b) / n
    gm = min(grid_ms_by, key=grid_ms_by.get)
    del Gt
    degrid_ms_by = {}
    for m in (0, 9):
        pm = p_fix.replace(grid_method=m)
        for _ in range(2):
            wp.degrid(pm, wk, uvw, X, out=dout, ws=dws)
        torch.cuda.synchronize()
        a.record()
        for _ in range(n):
            wp.degrid(pm, wk, uvw, X, out=dout, ws=dws)
        b.record()
        torch.cuda.synchronize()
        degrid_ms_by[m] = a.elapsed_time(b) / n
    dm = min(degrid_ms_by, key=degrid_ms_by.get)
    del X, dws, dout
    pr = Predictor(p_fix.replace(grid_method=gm), planes.cpu().numpy(), sup.cpu().tolist(), uvw, degrid_method=dm)
    # model image: the sky's point sources on their pixels (non-zero, so that the taper enters)
    img0 = torch.zeros((N, N), dtype=torch.float32)
    for l_, m_, f_ in zip(d["sky"].l, d["sky"].m, d["sky"].flux):
        img0[int(round(m_ / dl)) + N // 2, int(round(l_ / dl)) + N // 2] += float(f_)
    image = img0.to(dev).requires_grad_(True)
    taper = taper0.clone().requires_grad_(True)

    def step():
        image.grad = None
        taper.grad = None
        loss = chi2(pr(image, taper), vobs)
        loss.backward()
        return loss

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    a.record()
    for _ in range(n):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    # degridding roofline: 8 flop per footprint tap of every visibility (FP32 ALU), as gridding
    sup_h = sup.cpu().numpy()
    pl = planes.cpu().numpy()
    aw = np.abs(d["uvw"][:, 2].astype(np.float64))
    idx = np.clip(np.searchsorted(pl, aw), 1, P - 1)
    lower = np.where(np.abs(aw - pl[idx - 1]) <= np.abs(pl[idx] - aw), idx - 1, idx)
    taps = float(np.sum((2 * sup_h[lower].astype(np.float64) + 1) ** 2))
    pk = getattr(args, "peaks", None) or {}
    fp32_peak = pk.get("fp32_fma_tflops") or 152 * 128 * 2 * 2.07e9 / 1e12
    degrid_ms = degrid_ms_by[dm]
    achieved = 8.0 * taps / (degrid_ms * 1e-3) / 1e12
    names = {0: "warp per visibility (grid_method 0)", 9: "slots in reverse (grid_method 9)"}
    return {"workload": f"{V} visibilities, 4096^2 float32 model image, 512 planes, 512-sample taper, chi^2",
            "ms_per_forward_backward": ms, "mvis_per_s": V / (ms * 1e-3) / 1e6,
            "grad_image_norm": float(image.grad.norm()), "grad_taper_norm": float(taper.grad.norm()),
            "gridder_backward": GRID_METHOD_NAMES[gm],
            "grid_ms_by_method": {GRID_METHOD_NAMES[m]: t for m, t in grid_ms_by.items()},
            "degrid_ms": degrid_ms, "degrid_method": names[dm],
            "degrid_ms_by_method": {names[m]: t for m, t in degrid_ms_by.items()},
            "degrid_taps_per_vis": taps / V,
            "degrid_roofline": {"kernel": "k_degrid" if dm == 0 else "k_degrid_slot", "bound": "alu",
                                "achieved": achieved, "peak": fp32_peak,
                                "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                                "peak_source": "measured in this run" if pk.get("fp32_fma_tflops") else "nominal"}}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed as it stands on the same workload, each step a
    bounded sample of 128 of the 512 planes (every fourth |w|), a few seconds of CPU work.
    value and ms_per_step are those of the sample actually run: kernels made / step time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_sample = 128
    step_s = []
    t0 = time.perf_counter()
    for s in range(args.warmup + args.steps):
        ts = time.perf_counter()
        rate, thr, sample = oracle_kernel_rate(n_planes=n_sample)
        if s >= args.warmup:
            step_s.append(time.perf_counter() - ts)
    total = time.perf_counter() - t0
    ms = float(np.mean(step_s)) * 1e3
    v = n_sample / (ms * 1e-3)
    sample = (f"{n_sample} of the 512 |w| planes per step (every fourth, supports 7..127), screen + "
              f"transform + spline + resample each; transform matrix excluded; value = {n_sample} kernels / "
              f"measured step time")
    out = {"metric": METRIC, "value": v, "unit": "w-kernels/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": "kernel-generation batch: 1024 signed w-planes linspace[-20000,20000] "
                                  "(512 distinct |w| kernels), R=4096, os=8, support 7..127 by |w|, "
                                  "4096^2 grid, 8 deg FOV, Gaussian taper sigma=0.3 FOV"},
           "cpu_baseline": {"value": v, "unit": "w-kernels/s", "cores": thr, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "w-kernels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": total}
    print(json.dumps(out))


def run_sweep(args):
    """Kernel-generation cost along the paper's scaling axes (its Figs. 3-7: number of
    w-planes, kernel support, oversampling, truncation level) on the headline geometry (4096^2,
    8 deg, R 4096, Gaussian taper, |w| linspace[0, 20000]), for the matrix Hankel route
    (TF32x3), the projection-slice Hankel route and the standard 2D-FFT route.  On the first
    three axes every plane takes the sweep's support; on the truncation axis each plane's
    support is the one its radial line gives at that level (S_max 255), the same supports
    for every route.  Each route's time covers the radial line (or the 2D transform) and the
    oversampled cache of every plane.  Prints one JSON line with the table."""
    import ctypes

    import torch

    import paper_1904_08463_gb300 as wp

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    dl = np.deg2rad(FOV_DEG) / N_IMG
    taper_d = torch.tensor(synth.gaussian_taper_samples(N_IMG, dl, R_KG), dtype=torch.float32, device=dev)
    lib = wp._lib.load()

    def timeit(fn, n):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    def point(P, S, os_, tau=0.0):
        plan = wp.Plan(N_IMG, dl, os_, S, 1, tau, R_KG, "cubic", "tf32x3")
        wpl = torch.tensor(np.linspace(0.0, 20000.0, P), dtype=torch.float64, device=dev)
        if tau > 0.0:
            # supports from the truncation rule on the radial lines (read back once, untimed)
            ws = wp.workspace(wp.kernelgen_workspace_bytes(plan, P), dev)
            wp.kernelgen_prepare(plan, P, ws)
            _, _, sup = wp.hankel_radial(plan, taper_d, wpl, ws)
            sup_h = [int(v) for v in sup.cpu()]
            del ws
        else:
            sup_h = [S] * P
            sup = torch.tensor(sup_h, dtype=torch.int32, device=dev)
        off_h = wp.kernel_layout(plan, sup_h)
        off = torch.tensor(off_h, dtype=torch.int64, device=dev)
        cache = torch.empty(off_h[-1], dtype=torch.complex64, device=dev)
        g = plan.geometry()
        radial = torch.empty((P, g.k_out), dtype=torch.complex64, device=dev)
        spl = torch.empty_like(radial)
        out = {"planes": P, "support": S, "oversampling": os_, "cache_gb": off_h[-1] * 8 / 1e9}
        if tau > 0.0:
            out.update(trunc_frac=tau, support_min=min(sup_h), support_mean=float(np.mean(sup_h)),
                       support_max=max(sup_h))
        for route in ("tf32x3", "projslice"):
            pr = plan.replace(kernelgen=route)
            ws = wp.workspace(wp.kernelgen_workspace_bytes(pr, P), dev)
            wp.kernelgen_prepare(pr, P, ws)

            # truncating routes recompute supports into scratch; the resample keeps the laid-out ones
            scratch = torch.empty_like(sup) if tau > 0.0 else None

            def run(pr=pr, ws=ws, scratch=scratch):
                wp.hankel_radial(pr, taper_d, wpl, ws, radial, spl, scratch)
                wp.resample(pr, radial, spl, sup, off, cache)

            out[route + "_ms"] = timeit(run, 5)
            del ws
        fws = wp.workspace(int(lib.wp_fft_workspace_bytes(ctypes.byref(plan.c()), P)), dev)

        def fft():
            wp._lib.check("wp_fft_wkernels", lib.wp_fft_wkernels(
                ctypes.byref(plan.c()), ctypes.c_void_p(taper_d.data_ptr()), ctypes.c_void_p(wpl.data_ptr()), P,
                ctypes.c_void_p(sup.data_ptr()), ctypes.c_void_p(off.data_ptr()), 1,
                ctypes.c_void_p(fws.data_ptr()), fws.numel(), ctypes.c_void_p(cache.data_ptr()),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

        out["fft2d_ms"] = timeit(fft, 2)
        out["fft2d_over_tf32x3"] = out["fft2d_ms"] / out["tf32x3_ms"]
        out["fft2d_over_projslice"] = out["fft2d_ms"] / out["projslice_ms"]
        del fws, cache
        torch.cuda.empty_cache()
        log(f"sweep {out}")
        return out

    rows = []
    for P in (16, 64, 256, 1024):
        rows.append(dict(axis="planes", **point(P, 127, 8)))
    for S in (31, 63, 255, 511):
        rows.append(dict(axis="support", **point(64, S, 8)))
    for os_ in (1, 2, 4, 16):
        rows.append(dict(axis="oversampling", **point(64, 127, os_)))
    for tau in (1e-4, 1e-3, 1e-2, 1e-1):
        rows.append(dict(axis="truncation", **point(64, 255, 8, tau)))
    print(json.dumps({"sweep": "kernel generation: matrix Hankel (TF32x3), projection-slice Hankel, 2D FFT",
                      "geometry": "4096^2, 8 deg, R 4096, Gaussian taper, |w| linspace[0, 20000], all planes "
                                  "at the listed support (truncation axis: supports from the truncation "
                                  "rule, S_max 255)", "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--kernelgen", default="bf16x3", choices=["fp32", "tf32x3", "bf16x3", "bf16x6", "projslice"])
    ap.add_argument("--no-imaging", dest="imaging", action="store_false")
    ap.add_argument("--imaging-vis", type=int, default=1 << 23)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-routes", dest="routes", action="store_false",
                    help="skip timing the other kernel-generation routes (FP32 Hankel, 2D FFT)")
    ap.add_argument("--imaging-planes", type=int, default=512)
    ap.add_argument("--grid-shape", default="",
                    help="gridder 'method,tile' for the imaging workload instead of the autotuner's pick")
    ap.add_argument("--no-batch", dest="batch", action="store_false",
                    help="skip the batched uneven-problem workload")
    ap.add_argument("--no-grad", dest="grad", action="store_false",
                    help="skip forward + backward of the prediction (differentiation workload)")
    ap.add_argument("--batch-problems", type=int, default=48)
    ap.add_argument("--hankel-only", action="store_true",
                    help="profiling aid: time only screen + Hankel product + spline (no cache)")
    ap.add_argument("--plane-stride", type=int, default=1,
                    help="use every n-th |w| plane of the batch (small cases for profiling)")
    ap.add_argument("--sweep", action="store_true",
                    help="kernel-generation cost over planes / support / oversampling for the three routes")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
