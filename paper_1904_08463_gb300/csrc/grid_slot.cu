// Slot gridder (grid_method 9; Alg. 1 / Alg. 2 gridding step): register accumulation with the
// work distribution of Romein (ICS 2012, "An efficient work-distribution strategy for gridding
// radio-telescope data on GPUs"), fed by a sort of each plane's visibilities along a Morton
// curve of their grid cells instead of by baseline.
//
// Every tap of a (2S+1)^2 footprint whose corner is (x0, y0) lands on a distinct residue class
// (x mod W, y mod W), W = 2S+1.  A lane that owns the residue (a, b) -- a "slot" -- therefore
// has exactly one tap of every visibility of the plane: the cell x = x0 + ((a - x0) mod W)
// (same for y), tap offset (x - x0, y - y0).  It keeps that cell's sum in a register and writes
// it to the grid (one float2 reduction) only when a later visibility moves its cell, which for
// visibilities sorted along a Morton curve of their cells happens for a few percent of the
// taps.  The fast path -- a visibility whose footprint corner equals the previous one's, 58 %
// of the steps on the full-imaging workload -- is one address, one 8-byte tap load and four
// FMAs per slot, every lane busy whatever the support.
//
// Binning for this method: the usual FP64 decisions (bin_decide), a key (plane, Morton code of
// (iu, iv)) sorted by the library's radix sort, per-plane bounds of the sorted list, and one
// gathered record per visibility: footprint corner, corner mod W, sub-kernel offset with the
// conjugation flag, original index; the weighted value beside it.  Work item = (plane, chunk of
// up to SLOT_CHUNK consecutive visibilities, tile of the W x W slots: 32 x SLOT_ROWS, or
// 16 x 2 SLOT_ROWS for the last W mod 32 <= 16 columns), one warp per item, pulled from a queue.
#include <cuda_runtime.h>

#include "wp_internal.cuh"
#include "grid_slot.cuh"

namespace wp {


__device__ __forceinline__ uint32_t spread16(uint32_t v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Binning decisions and sort keys: key = plane << mb | Morton(iu, iv); a dropped visibility gets
// plane P (sorted after every kept one).  rec as k_bin's record; weight sum and drops reduced.
__global__ void __launch_bounds__(256) k_bin_slot(int64_t V, const float* __restrict__ uvw, int P,
                                                  const double* __restrict__ w_planes,
                                                  const int32_t* __restrict__ support, int N, double du, int os,
                                                  int mb, const float* __restrict__ weight,
                                                  uint64_t* __restrict__ keys, uint32_t* __restrict__ idx,
                                                  int4* __restrict__ rec, double* __restrict__ red) {
    extern __shared__ double wps[];
    __shared__ double red_w[8];
    __shared__ double red_d[8];
    for (int i = threadIdx.x; i < P; i += blockDim.x) wps[i] = w_planes[i];
    __syncthreads();
    double wsum = 0.0, drops = 0.0;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < V) {
        int p, iu, iv, fu, fv, conj;
        const bool ok = bin_decide(uvw, k, P, wps, support, N, du, os, &p, &iu, &iv, &fu, &fv, &conj);
        if (ok) {
            keys[k] = ((uint64_t)p << mb) | (uint64_t)(spread16((uint32_t)iu) | (spread16((uint32_t)iv) << 1));
            rec[k] = make_int4(iu | (iv << 16), fu | (fv << 8) | (conj << 16), p, (int)k);
            wsum = weight ? (double)weight[k] : 1.0;
        } else {
            keys[k] = (uint64_t)P << mb;
            drops = 1.0;
        }
        idx[k] = (uint32_t)k;
    }
    for (int o = 16; o; o >>= 1) {
        wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
        drops += __shfl_xor_sync(0xffffffffu, drops, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red_w[wid] = wsum; red_d[wid] = drops; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red_w[q]; b += red_d[q]; }
        if (a != 0.0) atomicAdd(&red[0], a);
        if (b != 0.0) atomicAdd(&red[1], b);
    }
}

// vstart[q] = first sorted position of plane q (q = 0..P; vstart[P] = number kept).  Each
// position where the plane changes writes the starts of the planes it steps over.
__global__ void __launch_bounds__(256) k_plane_bounds(int64_t V, int P, int mb, const uint64_t* __restrict__ keys,
                                                      int* __restrict__ vstart) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (V == 0) {
        for (int q = (int)i; q <= P; q += blockDim.x * gridDim.x) vstart[q] = 0;
        return;
    }
    if (i >= V) return;
    const int pi = (int)(keys[i] >> mb);
    const int pprev = (i == 0) ? -1 : (int)(keys[i - 1] >> mb);
    for (int q = pprev + 1; q <= pi; ++q) vstart[q] = (int)i;
    if (i == V - 1)
        for (int q = pi + 1; q <= P; ++q) vstart[q] = (int)V;
}

__global__ void __launch_bounds__(256) k_gather_slot(int64_t V, int os, int s_max, const int* __restrict__ vstart, int P,
                                                     const uint32_t* __restrict__ idx, const int4* __restrict__ rec,
                                                     const int32_t* __restrict__ support,
                                                     const float2* __restrict__ vis, const float* __restrict__ weight,
                                                     int4* __restrict__ srec, float2* __restrict__ svis) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V || i >= vstart[P]) return;
    slot_gather_one(i, os, s_max, idx, rec, support, vis, weight, srec, svis);
}

// Items of plane q: ceil(n_q / SLOT_CHUNK) chunks x slot_tiles_mixed(W, rows) tiles (rows: the
// slot rows per lane of the walk that consumes the items).
__global__ void __launch_bounds__(256) k_plane_items(int P, int s_max, const int* __restrict__ vstart,
                                                     const int32_t* __restrict__ support, int rows,
                                                     int* __restrict__ icount) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > P) return;
    if (q == P) { icount[P] = 0; return; }
    const int n = vstart[q + 1] - vstart[q];
    const int W = 2 * min(max(support[q], 1), s_max) + 1;
    icount[q] = (n > 0) ? ((n + SLOT_CHUNK - 1) / SLOT_CHUNK) * slot_tiles_mixed(W, rows) : 0;
}

template <int ROWS>
__global__ void __launch_bounds__(SLOT_WARPS * 32, 3) k_grid_slot(int N, int P, int s_max,
                                                                  const int32_t* __restrict__ support,
                                                                  const int64_t* __restrict__ offsets,
                                                                  const float2* __restrict__ cache,
                                                                  const int* __restrict__ vstart,
                                                                  const int* __restrict__ istart,
                                                                  const int4* __restrict__ srec,
                                                                  const float2* __restrict__ svis,
                                                                  int* __restrict__ ctrl, float2* __restrict__ grid) {
    const int lane = threadIdx.x & 31;
    const int n_items = istart[P];
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&ctrl[0], 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        slot_item<ROWS, false>(it, N, P, s_max, support, offsets, cache, vstart, istart, srec, svis, grid);
    }
}

// Degridding with slots (grid_method 9): the adjoint walk -- each slot holds the grid value of
// its cell, reloaded only when the cell changes; per visibility and slot tile the warp's sum of
// conj(tap) x value is added into vis_out (zeroed first) by lane 0.
template <int ROWS>
__global__ void __launch_bounds__(SLOT_WARPS * 32, 3) k_degrid_slot(int N, int P, int s_max,
                                                                    const int32_t* __restrict__ support,
                                                                    const int64_t* __restrict__ offsets,
                                                                    const float2* __restrict__ cache,
                                                                    const int* __restrict__ vstart,
                                                                    const int* __restrict__ istart,
                                                                    const int4* __restrict__ srec,
                                                                    const float2* __restrict__ grid,
                                                                    int* __restrict__ ctrl, float2* __restrict__ vis_out,
                                                                    int64_t V) {
    const int lane = threadIdx.x & 31;
    const int n_items = istart[P];
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&ctrl[0], 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        slot_item<ROWS, false, true>(it, N, P, s_max, support, offsets, cache, vstart, istart, srec, nullptr,
                                     const_cast<float2*>(grid), vis_out, V);
    }
}

static int bits_for(int64_t n) {       // bits to hold values 0 .. n - 1 (at least 1)
    int b = 1;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

size_t slot_hist_ints(int64_t V) { return radix_sort_hist_ints(V); }

int grid_slot(const Geom& g, const wp_wkernels* kern, const float* uvw, const float2* vis, const float* weight,
              int64_t V, const GridWork& w, float2* grid, double* stats, cudaStream_t st) {
    const int P = kern->P;
    const uint32_t* idx = nullptr;
    int rc = grid_slot_prepare(g, kern, uvw, weight, V, w, st, &idx, false);
    if (rc) return rc;
    if (V > 0) {
        k_gather_slot<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(V, g.os, g.s_max, w.vstart, P, idx, w.rec, w.seff,
                                                                   vis, weight, w.srec, w.svis);
        WP_LAUNCH_CHECK("k_gather_slot");
    }
    int dev = 0, sms = 0, per_sm = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_slot<SLOT_ROWS>, SLOT_WARPS * 32, 0));
    if (per_sm < 1) per_sm = 1;
    k_grid_slot<SLOT_ROWS><<<sms * per_sm, SLOT_WARPS * 32, 0, st>>>(g.N, P, g.s_max, w.seff, kern->offsets,
                                                          reinterpret_cast<const float2*>(kern->cache), w.vstart,
                                                          w.istart, w.srec, w.svis, w.ctrl, grid);
    WP_LAUNCH_CHECK("k_grid_slot");
    return stats ? add_stats(stats, w.red, st) : WP_OK;
}

// Binning of the slot gridder up to its item list: effective supports, decisions and keys, the
// sort, plane bounds, item counts and their scan; *idx_sorted = the sort's permutation.  The gather
// of the sorted records (k_gather_slot / slot_gather_one) is left to the caller.
int grid_slot_prepare(const Geom& g, const wp_wkernels* kern, const float* uvw, const float* weight, int64_t V,
                      const GridWork& w, cudaStream_t st, const uint32_t** idx_sorted, bool degrid) {
    // the slot rows per lane of the walk that will consume the items
    const int P = kern->P;
    int rc = WP_OK;
    WP_CUDA(cudaMemsetAsync(w.ctrl, 0, sizeof(int) * 8, st));
    WP_CUDA(cudaMemsetAsync(w.red, 0, sizeof(double) * 2, st));
    k_fit_supports_launch(g, kern, w, st);
    WP_LAUNCH_CHECK("k_fit_supports");
    const int mb = 2 * bits_for(g.N);
    const int bits = mb + bits_for((int64_t)P + 1);
    if (V > 0) {
        size_t smem = (size_t)P * sizeof(double);
        if (smem > 48 * 1024)
            WP_CUDA(cudaFuncSetAttribute(k_bin_slot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_bin_slot<<<(unsigned)((V + 255) / 256), 256, smem, st>>>(V, uvw, P, kern->w_planes, w.seff, g.N, g.du, g.os,
                                                                  mb, weight, w.skey, w.sidx, w.rec, w.red);
        WP_LAUNCH_CHECK("k_bin_slot");
    }
    bool in_alt = false;
    rc = radix_sort<uint64_t>(w.skey, w.sidx, w.skey_alt, w.sidx_alt, V, bits, w.rs_hist, w.rs_tmp, st, &in_alt);
    if (rc) return rc;
    const uint64_t* keys = in_alt ? w.skey_alt : w.skey;
    const uint32_t* idx = in_alt ? w.sidx_alt : w.sidx;
    k_plane_bounds<<<(unsigned)(V > 0 ? (V + 255) / 256 : 1), 256, 0, st>>>(V, P, mb, keys, w.vstart);
    WP_LAUNCH_CHECK("k_plane_bounds");
    k_plane_items<<<(unsigned)((P + 1 + 255) / 256), 256, 0, st>>>(P, g.s_max, w.vstart, w.seff,
                                                                    degrid ? SLOT_DEGRID_ROWS : SLOT_ROWS, w.icount);
    WP_LAUNCH_CHECK("k_plane_items");
    rc = exclusive_scan_i32(w.icount, w.istart, (int64_t)P + 1, w.scan_tmp, st);
    if (rc) return rc;
    *idx_sorted = idx;
    return WP_OK;
}

int degrid_slot(const Geom& g, const wp_wkernels* kern, const float* uvw, int64_t V, const GridWork& w,
                const float2* grid, float2* vis_out, cudaStream_t st) {
    const int P = kern->P;
    WP_CUDA(cudaMemsetAsync(vis_out, 0, sizeof(float2) * (size_t)V, st));
    const uint32_t* idx = nullptr;
    int rc = grid_slot_prepare(g, kern, uvw, nullptr, V, w, st, &idx, true);
    if (rc) return rc;
    if (V == 0) return WP_OK;
    k_gather_slot<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(V, g.os, g.s_max, w.vstart, P, idx, w.rec, w.seff,
                                                               nullptr, nullptr, w.srec, nullptr);
    WP_LAUNCH_CHECK("k_gather_slot");
    int dev = 0, sms = 0, per_sm = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_degrid_slot<SLOT_DEGRID_ROWS>, SLOT_WARPS * 32, 0));
    if (per_sm < 1) per_sm = 1;
    k_degrid_slot<SLOT_DEGRID_ROWS><<<sms * per_sm, SLOT_WARPS * 32, 0, st>>>(g.N, P, g.s_max, w.seff, kern->offsets,
                                                            reinterpret_cast<const float2*>(kern->cache), w.vstart,
                                                            w.istart, w.srec, grid, w.ctrl, vis_out, V);
    WP_LAUNCH_CHECK("k_degrid_slot");
    return WP_OK;
}

}  // namespace wp
