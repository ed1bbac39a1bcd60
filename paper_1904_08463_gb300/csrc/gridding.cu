// Convolutional gridding with w-projection kernels (Alg. 1 / Alg. 2 gridding step) and
// its adjoint, degridding.
//
//   K9  bin      per visibility: nearest |w| plane, conjugation flag (w < 0, Section 4.1),
//                grid cell + oversampling offset, drop test; all decisions in FP64
//   --  sort     counting sort by (plane, T x T centre tile; T = 64 or 32): histogram, scan,
//                scatter (uv-sorted binning: consecutive records share a plane and a tile)
//   --  items    work items (plane, output tile) that some visibility's footprint reaches
//   K10 grid     persistent blocks pull work items in plane-major order and own one T x T
//                output tile each, flushed once per item (one float2 atomic per touched
//                cell).  Five shapes, equal up to FP32 summation order, picked per problem
//                class by the autotuner:
//                  0 register tile: warp w owns rows (T/8) w .., lane l columns l, l+32, ..;
//                    every warp walks the neighbouring bins' visibilities on its own
//                  1 shared-memory tile, each warp takes whole visibilities and spreads the
//                    footprint over its lanes (shared float atomics)
//                  2 per-warp shared-memory 32 x 32 tiles over groups of 8 planes
//                  3 shared-memory tile; the block decodes the candidates once into a
//                    compact list of those that meet the tile, and warp w updates only rows
//                    w, w + 8, .. (plain read-modify-write, no atomics) -- the fastest
//                  4 as 3, each tap interpolated from the plane's radial line (no cache)
//   K11 degrid   one warp per visibility gathers conj(tap) x grid over the footprint and
//                reduces with shuffles
#include <cuda_runtime.h>
#include <math.h>

#include "wp_internal.cuh"
#include "grid_ro.cuh"

namespace wp {

namespace {
constexpr int SCAN_PER_BLOCK = 2048;
}  // namespace

// =======================================================================================
// exclusive scan of int32 (n values -> n values; callers append a zero to get the total)
// =======================================================================================
__global__ void __launch_bounds__(256) k_scan_block(const int* __restrict__ in, int* __restrict__ out,
                                                    int64_t n, int* __restrict__ block_sums) {
    __shared__ int warp_tot[8];
    const int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK + threadIdx.x * 8;
    int v[8];
    int s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        int64_t i = base + q;
        v[q] = (i < n) ? in[i] : 0;
        s += v[q];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int woff = 0, btot = 0;
    for (int q = 0; q < 8; ++q) {
        if (q < wid) woff += warp_tot[q];
        btot += warp_tot[q];
    }
    int run = woff + incl - s;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        int64_t i = base + q;
        if (i < n) out[i] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = btot;
}

__global__ void k_scan_add(int* __restrict__ out, int64_t n, const int* __restrict__ offs) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK;
    const int add = offs[blockIdx.x];
    for (int q = threadIdx.x; q < SCAN_PER_BLOCK; q += blockDim.x) {
        int64_t i = base + q;
        if (i < n) out[i] += add;
    }
}

size_t scan_tmp_ints(int64_t n) {
    size_t total = 0;
    while (n > 1) {
        int64_t nb = (n + SCAN_PER_BLOCK - 1) / SCAN_PER_BLOCK;
        total += 2 * (size_t)nb + 64;
        n = nb;
    }
    return total + 64;
}

int exclusive_scan_i32(const int* in, int* out, int64_t n, int* tmp, cudaStream_t st) {
    if (n <= 0) return WP_OK;
    int64_t nb = (n + SCAN_PER_BLOCK - 1) / SCAN_PER_BLOCK;
    int* sums = tmp;
    int* sums_scan = tmp + nb + 32;
    k_scan_block<<<(unsigned)nb, 256, 0, st>>>(in, out, n, sums);
    WP_LAUNCH_CHECK("k_scan_block");
    if (nb > 1) {
        int rc = exclusive_scan_i32(sums, sums_scan, nb, tmp + 2 * nb + 64, st);
        if (rc) return rc;
        k_scan_add<<<(unsigned)nb, 256, 0, st>>>(out, n, sums_scan);
        WP_LAUNCH_CHECK("k_scan_add");
    }
    return WP_OK;
}

// =======================================================================================
// K9: binning.  Record layout (int4): x = iu | iv << 16, y = fu | fv << 8 | conj << 16,
// z = plane, w = original index.  key = plane * ntiles + (iv / T) * ntx + iu / T, or -1.
// =======================================================================================
// Effective supports of a call: each plane's support clamped to [1, S_max] and, when the
// kernels read a cache, to what the plane's block of it holds (fit_support; 0 = unusable
// plane).  Binning, the work items and every gridding / degridding kernel read this array,
// so a caller's inconsistent layout gives that plane smaller footprints (its visibilities are
// dropped when it holds none) but no access outside its block -- and the kernels themselves
// carry no extra control flow.
__global__ void __launch_bounds__(256) k_fit_supports(int P, int os, int s_max, const int32_t* __restrict__ support,
                                                      const int64_t* __restrict__ offsets, int* __restrict__ seff) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int S = min(max(support[p], 1), s_max);
    seff[p] = offsets ? fit_support(S, os, offsets, p) : S;
}

__global__ void __launch_bounds__(256) k_bin(int64_t V, const float* __restrict__ uvw, int P,
                                             const double* __restrict__ w_planes,
                                             const int32_t* __restrict__ support, int s_max, int N,
                                             double du, int os, int T, int ntx, int ntiles,
                                             const float* __restrict__ weight,
                                             int* __restrict__ key, int4* __restrict__ rec,
                                             int* __restrict__ count, double* __restrict__ red) {
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
            int kk = p * ntiles + (iv / T) * ntx + (iu / T);
            key[k] = kk;
            rec[k] = make_int4(iu | (iv << 16), fu | (fv << 8) | (conj << 16), p, (int)k);
            atomicAdd(&count[kk], 1);
            wsum = weight ? (double)weight[k] : 1.0;
        } else {
            key[k] = -1;
            drops = 1.0;
        }
    }
    // block reduction of the statistics, one double atomic per block
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

__global__ void __launch_bounds__(256) k_scatter(int64_t V, const int* __restrict__ key,
                                                 const int4* __restrict__ rec, const float2* __restrict__ vis,
                                                 const float* __restrict__ weight, const int* __restrict__ start,
                                                 int* __restrict__ cursor, int4* __restrict__ srec,
                                                 float2* __restrict__ svis) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V) return;
    int kk = key[k];
    if (kk < 0) return;
    int pos = start[kk] + atomicAdd(&cursor[kk], 1);
    srec[pos] = rec[k];
    if (svis) {
        float2 v = vis[k];
        float a = weight ? weight[k] : 1.0f;
        svis[pos] = make_float2(v.x * a, v.y * a);
    }
}

// Work-item flags: item (p, tile) is live if any centre tile within ceil(S_p / T) tiles
// holds a visibility of plane p (a footprint reaches at most that far).  Bin b's
// visibilities are [start[b], start[b+1]) of the sorted arrays (start[nbins] = total).
__global__ void __launch_bounds__(256) k_item_flags(int P, int T, int ntx, int ntiles, int s_max,
                                                    const int32_t* __restrict__ support,
                                                    const int* __restrict__ start, int* __restrict__ flags) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)P * ntiles;
    if (it >= n) { if (it == n) flags[n] = 0; return; }
    int p = (int)(it / ntiles);
    int t = (int)(it - (int64_t)p * ntiles);
    int oy = t / ntx, ox = t - oy * ntx;
    int D = (min(max(support[p], 1), s_max) + T - 1) / T;
    // `start` holds the exclusive scan of the per-bin counts, so a run of bins
    // [a, b] is non-empty iff start[b + 1] > start[a]
    const int* s = start + (int64_t)p * ntiles;
    const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
    int any = 0;
    for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy)
        any |= (s[cy * ntx + cx_hi + 1] > s[cy * ntx + cx_lo]);
    flags[it] = any;
}

__global__ void __launch_bounds__(256) k_item_write(int64_t n, const int* __restrict__ flags,
                                                    const int* __restrict__ pos, int* __restrict__ items,
                                                    int* __restrict__ ctrl) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it < n && flags[it]) items[pos[it]] = (int)it;
    if (it == n - 1) ctrl[1] = pos[it] + flags[it];
}

void k_fit_supports_launch(const Geom& g, const wp_wkernels* kern, const GridWork& w, cudaStream_t st) {
    k_fit_supports<<<(kern->P + 255) / 256, 256, 0, st>>>(kern->P, g.os, g.s_max, kern->support,
                                                         kern->cache ? kern->offsets : nullptr, w.seff);
}

int grid_bin(const Geom& g, const wp_wkernels* kern, const float* uvw, const float2* vis,
             const float* weight, int64_t V, const GridWork& w, cudaStream_t st) {
    int rc = grid_bin_noscatter(g, kern, uvw, weight, V, w, st);
    if (rc) return rc;
    if (V > 0) {
        unsigned blocks = (unsigned)((V + 255) / 256);
        k_scatter<<<blocks, 256, 0, st>>>(V, w.key, w.rec, vis, weight, w.count, w.cursor, w.srec,
                                          vis ? w.svis : nullptr);
        WP_LAUNCH_CHECK("k_scatter");
    }
    return WP_OK;
}

// Binning up to the scanned bin counts: records, keys, counts (no scatter into bin order).
int grid_bin_noscatter(const Geom& g, const wp_wkernels* kern, const float* uvw, const float* weight, int64_t V,
                       const GridWork& w, cudaStream_t st) {
    const int P = kern->P;
    WP_CUDA(cudaMemsetAsync(w.count, 0, sizeof(int) * (size_t)(w.nbins + 1), st));
    WP_CUDA(cudaMemsetAsync(w.cursor, 0, sizeof(int) * (size_t)w.nbins, st));
    WP_CUDA(cudaMemsetAsync(w.ctrl, 0, sizeof(int) * 8, st));
    WP_CUDA(cudaMemsetAsync(w.red, 0, sizeof(double) * 2, st));
    k_fit_supports<<<(P + 255) / 256, 256, 0, st>>>(P, g.os, g.s_max, kern->support,
                                                   kern->cache ? kern->offsets : nullptr, w.seff);
    WP_LAUNCH_CHECK("k_fit_supports");
    if (V > 0) {
        unsigned blocks = (unsigned)((V + 255) / 256);
        size_t smem = (size_t)P * sizeof(double);
        if (smem > 48 * 1024)
            WP_CUDA(cudaFuncSetAttribute(k_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_bin<<<blocks, 256, smem, st>>>(V, uvw, P, kern->w_planes, w.seff, g.s_max, g.N, g.du,
                                         g.os, w.T, w.ntx, w.ntiles, weight, w.key, w.rec, w.count, w.red);
        WP_LAUNCH_CHECK("k_bin");
    }
    return exclusive_scan_i32(w.count, w.count, w.nbins + 1, w.scan_tmp, st);
}

// Flags of the per-plane work items (plane, tile) into w.flags[0 .. P * ntiles] (last = 0).
int item_flags(const Geom& g, const wp_wkernels* kern, const GridWork& w, cudaStream_t st) {
    const int64_t n = (int64_t)kern->P * w.ntiles;
    k_item_flags<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(kern->P, w.T, w.ntx, w.ntiles, g.s_max, w.seff,
                                                                 w.count, w.flags);
    WP_LAUNCH_CHECK("k_item_flags");
    return WP_OK;
}

// =======================================================================================
// K10: gridding
// =======================================================================================
// One visibility's contribution to the warp's ROWS rows x COLS column groups.
template <int ROWS, int COLS>
__device__ __forceinline__ void grid_one(const int4 r4, const float2 vv, const float2* __restrict__ pcache,
                                         int os, int S, int W, int W2, int R0, int C0,
                                         float2 (&acc)[ROWS][COLS]) {
    const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
    const int ry0 = iv - S;
    if (ry0 > R0 + ROWS - 1 || ry0 + 2 * S < R0) return;
    const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
    const float sgn = (r4.y >> 16) ? -1.0f : 1.0f;
    const float2* sub = pcache + (int64_t)(fv * os + fu) * W2;
    int jx[COLS];
    bool vc[COLS];
#pragma unroll
    for (int c = 0; c < COLS; ++c) {
        jx[c] = C0 + 32 * c - (iu - S);
        vc[c] = (unsigned)jx[c] <= (unsigned)(2 * S);
    }
    float2 tp[ROWS][COLS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {                   // all loads first
        const int jy = R0 + r - ry0;
        const bool rv = (unsigned)jy <= (unsigned)(2 * S);
        const float2* row = sub + jy * W;
#pragma unroll
        for (int c = 0; c < COLS; ++c)
            tp[r][c] = (rv && vc[c]) ? __ldg(row + jx[c]) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int c = 0; c < COLS; ++c) {
            const float ti = sgn * tp[r][c].y;
            acc[r][c].x = fmaf(vv.x, tp[r][c].x, fmaf(-vv.y, ti, acc[r][c].x));
            acc[r][c].y = fmaf(vv.x, ti, fmaf(vv.y, tp[r][c].x, acc[r][c].y));
        }
}

template <int TILE>
__global__ void __launch_bounds__(GRID_WARPS * 32, 3) k_grid(int N, int os, int s_max, int ntx, int ntiles,
                                                          const int32_t* __restrict__ support,
                                                          const int64_t* __restrict__ offsets,
                                                          const float2* __restrict__ cache,
                                                          const int* __restrict__ start,
                                                          const int4* __restrict__ srec,
                                                          const float2* __restrict__ svis,
                                                          const int* __restrict__ items,
                                                          int* __restrict__ ctrl, float2* __restrict__ grid) {
    constexpr int ROWS = TILE / GRID_WARPS, COLS = TILE / 32;
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n_items = ctrl[1];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl[0], 1);
        __syncthreads();
        const int item_idx = s_item;
        __syncthreads();
        if (item_idx >= n_items) break;
        const int item = items[item_idx];
        const int p = item / ntiles;
        const int t = item - p * ntiles;
        const int oy = t / ntx, ox = t - oy * ntx;
        const int S = min(max(support[p], 1), s_max);
        const int W = 2 * S + 1;
        const int W2 = W * W;
        const int D = (S + TILE - 1) / TILE;
        const float2* pcache = cache + offsets[p];
        const int R0 = oy * TILE + wid * ROWS;
        const int C0 = ox * TILE + lane;
        float2 acc[ROWS][COLS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
#pragma unroll
            for (int c = 0; c < COLS; ++c) acc[r][c] = make_float2(0.f, 0.f);
        // every warp walks the same visibility list independently (records are read by all
        // lanes at once: one broadcast load each), so no block barrier inside the item
        const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
        for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy) {
            const int kb = p * ntiles + cy * ntx;
            const int beg = start[kb + cx_lo], end = start[kb + cx_hi + 1];
            int q = beg;
            for (; q + 1 < end; q += 2) {
                const int4 ra = __ldg(srec + q);
                const int4 rb = __ldg(srec + q + 1);
                const float2 va = __ldg(svis + q);
                const float2 vb = __ldg(svis + q + 1);
                grid_one<ROWS, COLS>(ra, va, pcache, os, S, W, W2, R0, C0, acc);
                grid_one<ROWS, COLS>(rb, vb, pcache, os, S, W, W2, R0, C0, acc);
            }
            if (q < end) grid_one<ROWS, COLS>(__ldg(srec + q), __ldg(svis + q), pcache, os, S, W, W2, R0, C0, acc);
        }
        // flush the tile: one atomic per touched cell
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int row = R0 + r;
            if (row >= N) continue;
#pragma unroll
            for (int c = 0; c < COLS; ++c) {
                const int col = C0 + 32 * c;
                if (col < N && (acc[r][c].x != 0.0f || acc[r][c].y != 0.0f))
                    atomicAdd(grid + (int64_t)row * N + col, acc[r][c]);
            }
        }
    }
}

// Footprint-major variant: the block's T x T output tile lives in shared memory; each warp
// takes whole visibilities (round robin over the item's list) and spreads the footprint's
// intersection with the tile over its 32 lanes as one flat index range, so every lane does
// a useful tap whatever the support; contributions from different warps meet in shared
// memory through float atomics, and the tile is flushed once per item.
template <int TILE>
__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid_fm(int N, int os, int s_max, int ntx, int ntiles,
                                                             const int32_t* __restrict__ support,
                                                             const int64_t* __restrict__ offsets,
                                                             const float2* __restrict__ cache,
                                                             const int* __restrict__ start,
                                                             const int4* __restrict__ srec,
                                                             const float2* __restrict__ svis,
                                                             const int* __restrict__ items,
                                                             int* __restrict__ ctrl, float2* __restrict__ grid) {
    constexpr int TP = TILE + 1;                  // padded row: row wraps land on other banks
    __shared__ float tre[TILE * TP];              // real and imaginary parts in separate planes:
    __shared__ float tim[TILE * TP];              // consecutive lanes hit consecutive banks
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n_items = ctrl[1];
    for (int i = threadIdx.x; i < TILE * TP; i += blockDim.x) { tre[i] = 0.0f; tim[i] = 0.0f; }
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl[0], 1);
        __syncthreads();
        const int item_idx = s_item;
        __syncthreads();
        if (item_idx >= n_items) break;
        const int item = items[item_idx];
        const int p = item / ntiles;
        const int t = item - p * ntiles;
        const int oy = t / ntx, ox = t - oy * ntx;
        const int S = min(max(support[p], 1), s_max);
        const int W = 2 * S + 1;
        const int W2 = W * W;
        const int D = (S + TILE - 1) / TILE;
        const float2* pcache = cache + offsets[p];
        const int ty0 = oy * TILE, tx0 = ox * TILE;
        const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
        int seq = 0;   // position in the item's visibility list (same on every warp)
        for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy) {
            const int kb = p * ntiles + cy * ntx;
            const int beg = start[kb + cx_lo], end = start[kb + cx_hi + 1];
            const int first = beg + ((wid - seq) % GRID_WARPS + GRID_WARPS) % GRID_WARPS;
            seq += end - beg;
            for (int q = first; q < end; q += GRID_WARPS) {
                const int4 r4 = __ldg(srec + q);
                const float2 vv = __ldg(svis + q);
                const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
                // intersection of the footprint [iu-S, iu+S] x [iv-S, iv+S] with the tile
                const int c0 = max(iu - S, tx0), c1 = min(iu + S, tx0 + TILE - 1);
                const int r0 = max(iv - S, ty0), r1 = min(iv + S, ty0 + TILE - 1);
                if (c0 > c1 || r0 > r1) continue;
                const int w = c1 - c0 + 1, h = r1 - r0 + 1;
                const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
                const float sgn = (r4.y >> 16) ? -1.0f : 1.0f;
                const float2* sub = pcache + (int64_t)(fv * os + fu) * W2 + (r0 - (iv - S)) * W + (c0 - (iu - S));
                const int tbase = (r0 - ty0) * TP + (c0 - tx0);
                // lane-strided walk over the h x w rectangle, rows followed incrementally
                const int step_r = 32 / w, step_c = 32 - step_r * w;
                int row = lane / w, col = lane - (lane / w) * w;
                for (int i = lane; i < h * w; i += 32) {
                    const float2 tp = __ldg(sub + row * W + col);
                    const float ti = sgn * tp.y;
                    const int cell = tbase + row * TP + col;
                    atomicAdd(tre + cell, fmaf(vv.x, tp.x, -vv.y * ti));
                    atomicAdd(tim + cell, fmaf(vv.x, ti, vv.y * tp.x));
                    col += step_c;
                    row += step_r;
                    if (col >= w) { col -= w; ++row; }
                }
            }
        }
        __syncthreads();
        // flush the tile (one atomic per touched cell) and clear it for the next item
        for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
            const int ry = i / TILE, rx = i - ry * TILE;
            const int c = ry * TP + rx;
            const float2 a = make_float2(tre[c], tim[c]);
            if (a.x != 0.0f || a.y != 0.0f) {
                const int gy = ty0 + ry, gx = tx0 + rx;
                if (gy < N && gx < N) atomicAdd(grid + (int64_t)gy * N + gx, a);
                tre[c] = 0.0f;
                tim[c] = 0.0f;
            }
        }
    }
}

// Row-owned shared tile (grid_method 3): the block's TILE x TILE output tile lives in shared
// memory.  The item's candidate visibilities (the bins within footprint reach) are first
// decoded by the whole block, one candidate per thread, into a compact shared list of those
// whose footprint meets the tile (intersection rectangle, first tap, weighted value, conj
// flag).  Every warp then walks that list but touches only the tile rows it owns (row r
// belongs to warp r mod GRID_WARPS), its lanes across the intersection's columns.  Two warps
// never touch the same cell and neither do two lanes, so the accumulation is a plain
// shared-memory read-modify-write: no atomics, no private copies, and a visibility is decoded
// once per block rather than once per warp.

template <int TILE>
__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid_ro(int N, int os, int s_max, int ntx, int ntiles,
                                                             const int32_t* __restrict__ support,
                                                             const int64_t* __restrict__ offsets,
                                                             const float2* __restrict__ cache,
                                                             const int* __restrict__ start,
                                                             const int4* __restrict__ srec,
                                                             const float2* __restrict__ svis,
                                                             const int* __restrict__ items,
                                                             int* __restrict__ ctrl, float2* __restrict__ grid) {
    __shared__ float2 tile[TILE * TILE];
    __shared__ int l_off[RO_LIST];                // first tap of the intersection in the plane's cache
    __shared__ uint32_t l_geo[RO_LIST];           // r0 | r1 << 8 | c0 << 16 | (w - 1) << 24 | conj << 31
    __shared__ float2 l_vv[RO_LIST];
    __shared__ int s_item, s_n;
    const int n_items = ctrl[1];
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) tile[i] = make_float2(0.0f, 0.0f);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl[0], 1);
        __syncthreads();
        const int item_idx = s_item;
        __syncthreads();
        if (item_idx >= n_items) break;
        const int item = items[item_idx];
        ro_item<TILE, false>(item, N, os, s_max, ntx, ntiles, support, offsets, cache, start, srec, svis, grid,
                             tile, l_off, l_geo, l_vv, &s_n);
    }
}

// Row-owned shared tile with B entries per read-modify-write (grid_method 7: B = 2, 8: B = 4).
// Method 3 pays, per tap, an 8-byte tap load and a 16-byte shared read-modify-write, all through
// the L1 data path, which bounds it.  Here the candidates are compacted into the list in bin
// order (a ballot per warp, so consecutive entries are consecutive visibilities of the bin --
// usually the same baseline a few dumps apart, with nearly the same rectangle), and each warp
// takes B consecutive entries at a time: over the union of their rectangles restricted to its
// rows, every lane loads the taps of the entries that cover its cell and applies all of them in
// one read-modify-write, so the shared traffic per tap drops by up to B.
template <int TILE, int B>
__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid_rb(int N, int os, int s_max, int ntx, int ntiles,
                                                             const int32_t* __restrict__ support,
                                                             const int64_t* __restrict__ offsets,
                                                             const float2* __restrict__ cache,
                                                             const int* __restrict__ start,
                                                             const int4* __restrict__ srec,
                                                             const float2* __restrict__ svis,
                                                             const int* __restrict__ items,
                                                             int* __restrict__ ctrl, float2* __restrict__ grid) {
    constexpr int CH = TILE / 32;                 // column chunks of a tile row
    __shared__ float2 tile[TILE * TILE];
    __shared__ int l_off[RO_LIST];                // first tap of the intersection in the plane's cache
    __shared__ uint32_t l_geo[RO_LIST];           // r0 | r1 << 8 | c0 << 16 | c1 << 24 (tile coordinates)
    __shared__ float4 l_cf[RO_LIST];              // (Re V, -s Im V, s Re V, Im V), s = -1 for w < 0
    __shared__ int s_wcnt[GRID_WARPS];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int n_items = ctrl[1];
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) tile[i] = make_float2(0.0f, 0.0f);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl[0], 1);
        __syncthreads();
        const int item_idx = s_item;
        __syncthreads();
        if (item_idx >= n_items) break;
        const int item = items[item_idx];
        const int p = item / ntiles;
        const int t = item - p * ntiles;
        const int oy = t / ntx, ox = t - oy * ntx;
        const int S = min(max(support[p], 1), s_max);
        const int W = 2 * S + 1;
        const int W2 = W * W;
        const int D = (S + TILE - 1) / TILE;
        const float2* pcache = cache + offsets[p];
        const int ty0 = oy * TILE, tx0 = ox * TILE;
        const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
        for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy) {
            const int kb = p * ntiles + cy * ntx;
            const int beg = start[kb + cx_lo], end = start[kb + cx_hi + 1];
            for (int base = beg; base < end; base += RO_LIST) {
                // decode one candidate per thread; compact in bin order (ballot + warp offsets)
                const int q = base + (int)threadIdx.x;
                int iu = 0, iv = 0, c0 = 0, c1 = -1, r0 = 0, r1 = -1;
                int4 r4 = make_int4(0, 0, 0, 0);
                if (q < end) {
                    r4 = __ldg(srec + q);
                    iu = r4.x & 0xffff;
                    iv = (r4.x >> 16) & 0xffff;
                    c0 = max(iu - S, tx0);
                    c1 = min(iu + S, tx0 + TILE - 1);
                    r0 = max(iv - S, ty0);
                    r1 = min(iv + S, ty0 + TILE - 1);
                }
                const bool meets = c0 <= c1 && r0 <= r1;
                const unsigned bal = __ballot_sync(0xffffffffu, meets);
                if (lane == 0) s_wcnt[wid] = __popc(bal);
                __syncthreads();
                int woff = 0, n = 0;
#pragma unroll
                for (int w = 0; w < GRID_WARPS; ++w) {
                    const int cw = s_wcnt[w];
                    woff += (w < wid) ? cw : 0;
                    n += cw;
                }
                if (meets) {
                    const int slot = woff + __popc(bal & lt);
                    const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
                    const float sg = ((r4.y >> 16) & 1) ? -1.0f : 1.0f;
                    const float2 vv = __ldg(svis + q);
                    l_off[slot] = (fv * os + fu) * W2 + (r0 - (iv - S)) * W + (c0 - (iu - S));
                    l_geo[slot] = (uint32_t)(r0 - ty0) | ((uint32_t)(r1 - ty0) << 8) |
                                  ((uint32_t)(c0 - tx0) << 16) | ((uint32_t)(c1 - tx0) << 24);
                    l_cf[slot] = make_float4(vv.x, -sg * vv.y, sg * vv.x, vv.y);
                }
                __syncthreads();
                for (int e0 = 0; e0 < n; e0 += B) {
                    int br0[B], br1[B], bc0[B], bc1[B], boff[B];
                    float4 bcf[B];
                    int R0 = TILE, R1 = -1, C0 = TILE, C1 = -1;
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        if (e0 + b < n) {
                            const uint32_t geo = l_geo[e0 + b];
                            br0[b] = (int)(geo & 0xff);
                            br1[b] = (int)((geo >> 8) & 0xff);
                            bc0[b] = (int)((geo >> 16) & 0xff);
                            bc1[b] = (int)(geo >> 24);
                            boff[b] = l_off[e0 + b] - br0[b] * W - bc0[b];   // tap of tile cell (0, 0)
                            bcf[b] = l_cf[e0 + b];
                        } else {
                            br0[b] = TILE; br1[b] = -1; bc0[b] = TILE; bc1[b] = -1; boff[b] = 0;
                            bcf[b] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        }
                        R0 = min(R0, br0[b]);
                        R1 = max(R1, br1[b]);
                        C0 = min(C0, bc0[b]);
                        C1 = max(C1, bc1[b]);
                    }
                    const int rw = R0 + ((wid - R0) & (GRID_WARPS - 1));   // first owned row
                    for (int r = rw; r <= R1; r += GRID_WARPS) {
                        float2* trow = tile + r * TILE;
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            const int c = C0 + lane + 32 * k;
                            if (c <= C1) {
                                float2 tp[B];
#pragma unroll
                                for (int b = 0; b < B; ++b) {
                                    const bool v = r >= br0[b] && r <= br1[b] && c >= bc0[b] && c <= bc1[b];
                                    tp[b] = v ? __ldg(pcache + (boff[b] + r * W + c)) : make_float2(0.0f, 0.0f);
                                }
                                float2 a = trow[c];
#pragma unroll
                                for (int b = 0; b < B; ++b) {
                                    a.x = fmaf(bcf[b].x, tp[b].x, fmaf(bcf[b].y, tp[b].y, a.x));
                                    a.y = fmaf(bcf[b].z, tp[b].y, fmaf(bcf[b].w, tp[b].x, a.y));
                                }
                                trow[c] = a;
                            }
                        }
                    }
                    __syncwarp();   // the next entries may touch these cells from other lanes
                }
                __syncthreads();   // the list is rebuilt for the next round
            }
        }
        __syncthreads();
        // flush the tile (one atomic per touched cell) and clear it for the next item
        for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
            const float2 a = tile[i];
            if (a.x != 0.0f || a.y != 0.0f) {
                const int gy = ty0 + i / TILE, gx = tx0 + (i & (TILE - 1));
                if (gy < N && gx < N) atomicAdd(grid + (int64_t)gy * N + gx, a);
                tile[i] = make_float2(0.0f, 0.0f);
            }
        }
        __syncthreads();
    }
}

// On-the-fly taps (grid_method 4): the row-owned tile of method 3, but each tap is
// interpolated from the plane's radial line in shared memory (the resample's own evaluation,
// so the values are the cache's bits) instead of being read from the cache.  The line is
// staged once per run of consecutive items of the same plane.
template <int TILE, bool CUBIC>
__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid_otf(int N, int os, int s_max, int K, int ntx, int ntiles,
                                                              const int32_t* __restrict__ support,
                                                              const float2* __restrict__ radial,
                                                              const float2* __restrict__ spline_m,
                                                              const int* __restrict__ start,
                                                              const int4* __restrict__ srec,
                                                              const float2* __restrict__ svis,
                                                              const int* __restrict__ items,
                                                              int* __restrict__ ctrl, float2* __restrict__ grid) {
    constexpr int CH = TILE / 32;
    extern __shared__ float4 line[];              // skew(n_used) entries {y.re, y.im, m.re, m.im}
    __shared__ float2 tile[TILE * TILE];
    __shared__ int l_j[RO_LIST];                  // first footprint column | first row << 16
    __shared__ int l_f[RO_LIST];                  // fu | fv << 8
    __shared__ uint32_t l_geo[RO_LIST];           // r0 | r1 << 8 | c0 << 16 | (w - 1) << 24 | conj << 31
    __shared__ float2 l_vv[RO_LIST];
    __shared__ int s_item, s_n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n_items = ctrl[1];
    int line_p = -1;
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) tile[i] = make_float2(0.0f, 0.0f);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl[0], 1);
        __syncthreads();
        const int item_idx = s_item;
        __syncthreads();
        if (item_idx >= n_items) break;
        const int item = items[item_idx];
        const int p = item / ntiles;
        const int t = item - p * ntiles;
        const int oy = t / ntx, ox = t - oy * ntx;
        const int S = min(max(support[p], 1), s_max);
        const int lim = os * S, lim2 = lim * lim;
        if (p != line_p) {                        // block-uniform: every thread saw the same item
            const int n_used = min(K, lim + 2);
            const float2* yl = radial + (int64_t)p * K;
            const float2* ml = spline_m + (int64_t)p * K;
            for (int k = threadIdx.x; k < n_used; k += blockDim.x) {
                const float2 a = yl[k];
                const float2 b = CUBIC ? ml[k] : make_float2(0.0f, 0.0f);
                line[skew(k)] = make_float4(a.x, a.y, b.x, b.y);
            }
            line_p = p;
            __syncthreads();
        }
        const int D = (S + TILE - 1) / TILE;
        const int ty0 = oy * TILE, tx0 = ox * TILE;
        const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
        for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy) {
            const int kb = p * ntiles + cy * ntx;
            const int beg = start[kb + cx_lo], end = start[kb + cx_hi + 1];
            for (int base = beg; base < end; base += RO_LIST) {
                if (threadIdx.x == 0) s_n = 0;
                __syncthreads();
                const int q = base + (int)threadIdx.x;
                if (q < end) {
                    const int4 r4 = __ldg(srec + q);
                    const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
                    const int c0 = max(iu - S, tx0), c1 = min(iu + S, tx0 + TILE - 1);
                    const int r0 = max(iv - S, ty0), r1 = min(iv + S, ty0 + TILE - 1);
                    if (c0 <= c1 && r0 <= r1) {
                        const int slot = atomicAdd(&s_n, 1);
                        l_j[slot] = (c0 - (iu - S)) | ((r0 - (iv - S)) << 16);
                        l_f[slot] = r4.y & 0xffff;
                        l_geo[slot] = (uint32_t)(r0 - ty0) | ((uint32_t)(r1 - ty0) << 8) |
                                      ((uint32_t)(c0 - tx0) << 16) | ((uint32_t)(c1 - c0) << 24) |
                                      ((uint32_t)((r4.y >> 16) & 1) << 31);
                        l_vv[slot] = __ldg(svis + q);
                    }
                }
                __syncthreads();
                const int n = s_n;
                for (int e = 0; e < n; ++e) {
                    const uint32_t geo = l_geo[e];
                    const int r0 = (int)(geo & 0xff), r1 = (int)((geo >> 8) & 0xff);
                    const int rw = r0 + ((wid - r0) & (GRID_WARPS - 1));   // first owned row
                    if (rw > r1) continue;
                    const int c0 = (int)((geo >> 16) & 0xff), w = (int)((geo >> 24) & 0x7f) + 1;
                    const float sgn = (geo >> 31) ? -1.0f : 1.0f;
                    const float2 vv = l_vv[e];
                    const int jx0 = l_j[e] & 0xffff, jy0 = l_j[e] >> 16;
                    const int fu = l_f[e] & 0xff, fv = l_f[e] >> 8;
                    // fine offsets of the first tap of the intersection's first owned row
                    const int dx0 = os * (jx0 - S) - fu;
                    int dy = os * (jy0 + (rw - r0) - S) - fv;
                    float2* trow = tile + rw * TILE + c0;
                    for (int r = rw; r <= r1; r += GRID_WARPS) {
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            const int c = lane + 32 * k;
                            if (c < w) {
                                const float2 tp = resample_tap<CUBIC>(line, dx0 + os * c, dy, lim2);
                                const float ti = sgn * tp.y;
                                float2 a = trow[c];
                                a.x = fmaf(vv.x, tp.x, fmaf(-vv.y, ti, a.x));
                                a.y = fmaf(vv.x, ti, fmaf(vv.y, tp.x, a.y));
                                trow[c] = a;
                            }
                        }
                        dy += os * GRID_WARPS;
                        trow += GRID_WARPS * TILE;
                    }
                    __syncwarp();   // the next entry may touch this one's cells from other lanes
                }
                __syncthreads();   // the list is rebuilt for the next round
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
            const float2 a = tile[i];
            if (a.x != 0.0f || a.y != 0.0f) {
                const int gy = ty0 + i / TILE, gx = tx0 + (i & (TILE - 1));
                if (gy < N && gx < N) atomicAdd(grid + (int64_t)gy * N + gx, a);
                tile[i] = make_float2(0.0f, 0.0f);
            }
        }
        __syncthreads();
    }
}

// Warp-private variant (grid_method 2): 32 x 32 output tiles, one shared-memory copy of the
// tile per warp.  A work item is (group of PG consecutive planes, tile); each warp takes
// whole visibilities of the item's planes (round robin) and spreads the footprint's
// intersection with the tile over its lanes as one flat range -- distinct cells per lane, so
// a plain read-modify-write of the warp's own copy needs no atomics, and a visibility that
// misses the tile costs one warp a few instructions instead of every warp.  At the end of
// the item the copies are summed and the tile is flushed with one atomic per touched cell.
constexpr int WPT = 32;             // tile side of the warp-private variant
constexpr int WPT_PAD = WPT + 1;    // padded rows (row wraps of a lane range fall on other banks)
constexpr int PLANE_GROUP = 8;      // planes per work item

__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid_wp(int N, int os, int s_max, int P, int ntx, int ntiles,
                                                             const int32_t* __restrict__ support,
                                                             const int64_t* __restrict__ offsets,
                                                             const float2* __restrict__ cache,
                                                             const int* __restrict__ start,
                                                             const int4* __restrict__ srec,
                                                             const float2* __restrict__ svis,
                                                             const int* __restrict__ items,
                                                             int* __restrict__ ctrl, float2* __restrict__ grid) {
    extern __shared__ float smem[];                      // [GRID_WARPS][2][WPT * WPT_PAD]
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float* myre = smem + wid * 2 * WPT * WPT_PAD;
    float* myim = myre + WPT * WPT_PAD;
    for (int i = threadIdx.x; i < GRID_WARPS * 2 * WPT * WPT_PAD; i += blockDim.x) smem[i] = 0.0f;
    const int n_items = ctrl[1];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl[0], 1);
        __syncthreads();
        const int item_idx = s_item;
        __syncthreads();
        if (item_idx >= n_items) break;
        const int item = items[item_idx];
        const int grp = item / ntiles;
        const int t = item - grp * ntiles;
        const int oy = t / ntx, ox = t - oy * ntx;
        const int ty0 = oy * WPT, tx0 = ox * WPT;
        int seq = 0;   // position in the item's visibility list (identical on every warp)
        for (int p = grp * PLANE_GROUP; p < min(P, (grp + 1) * PLANE_GROUP); ++p) {
            const int S = min(max(support[p], 1), s_max);
            const int W = 2 * S + 1, W2 = W * W;
            const int D = (S + WPT - 1) / WPT;
            const float2* pcache = cache + offsets[p];
            const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
            for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy) {
                const int kb = p * ntiles + cy * ntx;
                const int beg = start[kb + cx_lo], end = start[kb + cx_hi + 1];
                const int first = beg + ((wid - seq) % GRID_WARPS + GRID_WARPS) % GRID_WARPS;
                seq += end - beg;
                for (int q = first; q < end; q += GRID_WARPS) {
                    const int4 r4 = __ldg(srec + q);
                    const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
                    const int c0 = max(iu - S, tx0), c1 = min(iu + S, tx0 + WPT - 1);
                    const int r0 = max(iv - S, ty0), r1 = min(iv + S, ty0 + WPT - 1);
                    if (c0 > c1 || r0 > r1) continue;
                    const float2 vv = __ldg(svis + q);
                    const int w = c1 - c0 + 1, h = r1 - r0 + 1;
                    const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
                    const float sgn = (r4.y >> 16) ? -1.0f : 1.0f;
                    const float2* sub = pcache + (int64_t)(fv * os + fu) * W2 + (r0 - (iv - S)) * W + (c0 - (iu - S));
                    const int tb = (r0 - ty0) * WPT_PAD + (c0 - tx0);
                    const int step_r = 32 / w, step_c = 32 - step_r * w;
                    int row = lane / w, col = lane - (lane / w) * w;
                    for (int i = lane; i < h * w; i += 32) {
                        const float2 tp = __ldg(sub + row * W + col);
                        const float ti = sgn * tp.y;
                        const int cell = tb + row * WPT_PAD + col;
                        myre[cell] += fmaf(vv.x, tp.x, -vv.y * ti);
                        myim[cell] += fmaf(vv.x, ti, vv.y * tp.x);
                        col += step_c;
                        row += step_r;
                        if (col >= w) { col -= w; ++row; }
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        // sum the warp copies, flush, clear
        for (int i = threadIdx.x; i < WPT * WPT; i += blockDim.x) {
            const int ry = i / WPT, rx = i - ry * WPT;
            const int c = ry * WPT_PAD + rx;
            float ar = 0.0f, ai = 0.0f;
#pragma unroll
            for (int k = 0; k < GRID_WARPS; ++k) {
                float* b = smem + k * 2 * WPT * WPT_PAD;
                ar += b[c];
                ai += b[WPT * WPT_PAD + c];
                b[c] = 0.0f;
                b[WPT * WPT_PAD + c] = 0.0f;
            }
            if (ar != 0.0f || ai != 0.0f) {
                const int gy = ty0 + ry, gx = tx0 + rx;
                if (gy < N && gx < N) atomicAdd(grid + (int64_t)gy * N + gx, make_float2(ar, ai));
            }
        }
    }
}

// Work-item flags of the warp-private variant: (plane group, tile) is live if any plane of
// the group has a visibility within its footprint reach of the tile.
__global__ void __launch_bounds__(256) k_item_flags_grp(int P, int ngrp, int ntx, int ntiles, int s_max,
                                                        const int32_t* __restrict__ support,
                                                        const int* __restrict__ start, int* __restrict__ flags) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)ngrp * ntiles;
    if (it >= n) return;
    const int grp = (int)(it / ntiles);
    const int t = (int)(it - (int64_t)grp * ntiles);
    const int oy = t / ntx, ox = t - oy * ntx;
    int any = 0;
    for (int p = grp * PLANE_GROUP; p < min(P, (grp + 1) * PLANE_GROUP) && !any; ++p) {
        const int D = (min(max(support[p], 1), s_max) + WPT - 1) / WPT;
        const int* s = start + (int64_t)p * ntiles;
        const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
        for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy)
            any |= (s[cy * ntx + cx_hi + 1] > s[cy * ntx + cx_lo]);
    }
    flags[it] = any;
}

__global__ void k_add_stats(double* stats, const double* red) {
    if (threadIdx.x < 2) stats[threadIdx.x] += red[threadIdx.x];
}

int add_stats(double* stats, const double* red, cudaStream_t st) {
    k_add_stats<<<1, 32, 0, st>>>(stats, red);
    WP_LAUNCH_CHECK("k_add_stats");
    return WP_OK;
}

int write_items(int64_t n, const GridWork& w, cudaStream_t st) {
    k_item_write<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, w.flags, w.cursor, w.items, w.ctrl);
    WP_LAUNCH_CHECK("k_item_write");
    return WP_OK;
}

int grid_run(const Geom& g, const wp_wkernels* kern, const GridWork& w, float2* grid, double* stats,
             cudaStream_t st) {
    if (g.grid_method == 5 || g.grid_method == 6) {      // plane groups (grid_group.cu)
        int rc = grid_run_group(g, kern, w, grid, st);
        if (rc) return rc;
        return stats ? add_stats(stats, w.red, st) : WP_OK;
    }
    const int P = kern->P;
    const int ngrp = (P + PLANE_GROUP - 1) / PLANE_GROUP;
    const int64_t n = (g.grid_method == 2) ? (int64_t)ngrp * w.ntiles : (int64_t)P * w.ntiles;
    unsigned blocks = (unsigned)((n + 1 + 255) / 256);
    if (g.grid_method == 2)
        k_item_flags_grp<<<blocks, 256, 0, st>>>(P, ngrp, w.ntx, w.ntiles, g.s_max, w.seff, w.count, w.flags);
    else
        k_item_flags<<<blocks, 256, 0, st>>>(P, w.T, w.ntx, w.ntiles, g.s_max, w.seff, w.count, w.flags);
    WP_LAUNCH_CHECK("k_item_flags");
    // the flag scan reuses the cursor array as output (cursor is no longer needed)
    int rc = exclusive_scan_i32(w.flags, w.cursor, n, w.scan_tmp, st);
    if (rc) return rc;
    k_item_write<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, w.flags, w.cursor, w.items, w.ctrl);
    WP_LAUNCH_CHECK("k_item_write");
    int dev = 0, sms = 0, per_sm = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const float2* c2 = reinterpret_cast<const float2*>(kern->cache);
    if (g.grid_method == 2) {
        const size_t smem = (size_t)GRID_WARPS * 2 * WPT * WPT_PAD * sizeof(float);
        WP_CUDA(cudaFuncSetAttribute(k_grid_wp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_wp, GRID_WARPS * 32, smem));
        if (per_sm < 1) per_sm = 1;
        k_grid_wp<<<sms * per_sm, GRID_WARPS * 32, smem, st>>>(g.N, g.os, g.s_max, P, w.ntx, w.ntiles, w.seff,
                                                               kern->offsets, c2, w.count, w.srec, w.svis, w.items,
                                                               w.ctrl, grid);
    } else if (g.grid_method == 4) {
        int n_line = g.os * g.s_max + 2;
        if (n_line > g.k_out) n_line = g.k_out;
        n_line = (n_line + 7) / 8 * 8;
        const size_t smem = (size_t)n_line * sizeof(float4);
        const float2* rad = reinterpret_cast<const float2*>(kern->radial);
        const float2* spl = reinterpret_cast<const float2*>(kern->spline_m);
        const bool cubic = (g.interp == WP_INTERP_CUBIC);
#define WP_LAUNCH_OTF(T, C)                                                                                     \
        do {                                                                                                    \
            WP_CUDA(cudaFuncSetAttribute(k_grid_otf<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
            WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_otf<T, C>, GRID_WARPS * 32, smem)); \
            if (per_sm < 1) per_sm = 1;                                                                         \
            k_grid_otf<T, C><<<sms * per_sm, GRID_WARPS * 32, smem, st>>>(g.N, g.os, g.s_max, g.k_out, w.ntx,   \
                w.ntiles, w.seff, rad, spl, w.count, w.srec, w.svis, w.items, w.ctrl, grid);            \
        } while (0)
        if (w.T == 32) {
            if (cubic) WP_LAUNCH_OTF(32, true); else WP_LAUNCH_OTF(32, false);
        } else {
            if (cubic) WP_LAUNCH_OTF(64, true); else WP_LAUNCH_OTF(64, false);
        }
#undef WP_LAUNCH_OTF
    } else if (g.grid_method == 7 || g.grid_method == 8) {
#define WP_LAUNCH_RB(T, BB)                                                                                     \
        do {                                                                                                    \
            WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_rb<T, BB>, GRID_WARPS * 32, 0)); \
            if (per_sm < 1) per_sm = 1;                                                                         \
            k_grid_rb<T, BB><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, w.ntx, w.ntiles,     \
                w.seff, kern->offsets, c2, w.count, w.srec, w.svis, w.items, w.ctrl, grid);                     \
        } while (0)
        if (w.T == 32) {
            if (g.grid_method == 7) WP_LAUNCH_RB(32, 2); else WP_LAUNCH_RB(32, 4);
        } else {
            if (g.grid_method == 7) WP_LAUNCH_RB(64, 2); else WP_LAUNCH_RB(64, 4);
        }
#undef WP_LAUNCH_RB
    } else if (g.grid_method == 3) {
        if (w.T == 32) {
            WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_ro<32>, GRID_WARPS * 32, 0));
            if (per_sm < 1) per_sm = 1;
            k_grid_ro<32><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, w.ntx, w.ntiles,
                                                                    w.seff, kern->offsets, c2, w.count,
                                                                    w.srec, w.svis, w.items, w.ctrl, grid);
        } else {
            WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_ro<64>, GRID_WARPS * 32, 0));
            if (per_sm < 1) per_sm = 1;
            k_grid_ro<64><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, w.ntx, w.ntiles,
                                                                    w.seff, kern->offsets, c2, w.count,
                                                                    w.srec, w.svis, w.items, w.ctrl, grid);
        }
    } else if (g.grid_method == 1) {
        if (w.T == 32) {
            WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_fm<32>, GRID_WARPS * 32, 0));
            if (per_sm < 1) per_sm = 1;
            k_grid_fm<32><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, w.ntx, w.ntiles,
                                                                    w.seff, kern->offsets, c2, w.count,
                                                                    w.srec, w.svis, w.items, w.ctrl, grid);
        } else {
            WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_fm<64>, GRID_WARPS * 32, 0));
            if (per_sm < 1) per_sm = 1;
            k_grid_fm<64><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, w.ntx, w.ntiles,
                                                                    w.seff, kern->offsets, c2, w.count,
                                                                    w.srec, w.svis, w.items, w.ctrl, grid);
        }
    } else if (w.T == 32) {
        WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid<32>, GRID_WARPS * 32, 0));
        if (per_sm < 1) per_sm = 1;
        k_grid<32><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, w.ntx, w.ntiles, w.seff,
                                                             kern->offsets, c2, w.count, w.srec, w.svis, w.items,
                                                             w.ctrl, grid);
    } else {
        WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid<64>, GRID_WARPS * 32, 0));
        if (per_sm < 1) per_sm = 1;
        k_grid<64><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, w.ntx, w.ntiles, w.seff,
                                                             kern->offsets, c2, w.count, w.srec, w.svis, w.items,
                                                             w.ctrl, grid);
    }
    WP_LAUNCH_CHECK("k_grid");
    if (stats) {
        rc = add_stats(stats, w.red, st);
        if (rc) return rc;
    }
    return WP_OK;
}

// =======================================================================================
// K11: degridding (adjoint).  One warp per binned visibility.
// =======================================================================================
constexpr int DEGRID_UNROLL = 2;     // warp passes of 32 taps per loop trip of the degridder

__global__ void __launch_bounds__(256) k_degrid(int N, int os, int s_max, int nbins,
                                                const int32_t* __restrict__ support,
                                                const int64_t* __restrict__ offsets,
                                                const float2* __restrict__ cache, const int* __restrict__ start,
                                                const int4* __restrict__ srec, const float2* __restrict__ grid,
                                                float2* __restrict__ vis_out, int64_t V) {
    const int lane = threadIdx.x & 31;
    const int64_t wpos = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_valid = start[nbins];
    if (wpos >= n_valid || wpos >= V) return;
    const int4 r4 = srec[wpos];
    const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
    const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
    const float sgn = (r4.y >> 16) ? -1.0f : 1.0f;
    const int p = r4.z;
    const int S = min(max(support[p], 1), s_max);
    const int W = 2 * S + 1;
    const int64_t sb = (int64_t)(fv * os + fu) * W * W;
    const int64_t blk = offsets[p + 1] - offsets[p];   // the plane's block (checked build)
    const float2* sub = cache + offsets[p] + sb;
    const float2* g0 = grid + (int64_t)(iv - S) * N + (iu - S);
    const float2 zero = make_float2(0.0f, 0.0f);
    float sr = 0.0f, si = 0.0f;
    // The footprint's W^2 taps in storage order t = jy W + jx, 32 consecutive taps per warp pass
    // (every lane busy up to the last pass, whatever W), DEGRID_UNROLL passes per loop trip with
    // their tap and grid loads (L2) in flight together.  Lane position (jy, jx) of tap t advances
    // by 32 taps a pass: sy rows and sx columns, plus one row when the column wraps.
    const int W2 = W * W;
    const int sy = 32 / W, sx = 32 - sy * W;
    int jy = lane / W, jx = lane - (lane / W) * W;
    for (int t0 = 0; t0 < W2; t0 += 32 * DEGRID_UNROLL) {
        float2 tp[DEGRID_UNROLL], gv[DEGRID_UNROLL];
#pragma unroll
        for (int i = 0; i < DEGRID_UNROLL; ++i) {
            const int t = t0 + 32 * i + lane;
            const bool ok = t < W2;
            tp[i] = (ok && in_bounds(sb + t, blk, BS_TAP)) ? __ldg(sub + t) : zero;
            gv[i] = (ok && in_bounds(iu - S + jx, N, BS_GRID) && in_bounds(iv - S + jy, N, BS_GRID))
                        ? g0[(int64_t)jy * N + jx] : zero;
            jx += sx;
            jy += sy;
            if (jx >= W) { jx -= W; ++jy; }
        }
#pragma unroll
        for (int i = 0; i < DEGRID_UNROLL; ++i) {   // conj(K) * g
            const float ti = sgn * tp[i].y;
            sr = fmaf(tp[i].x, gv[i].x, fmaf(ti, gv[i].y, sr));
            si = fmaf(tp[i].x, gv[i].y, fmaf(-ti, gv[i].x, si));
        }
    }
    for (int o = 16; o; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0 && in_bounds(r4.w, V, BS_VIS)) vis_out[r4.w] = make_float2(sr, si);
}

int degrid_run(const Geom& g, const wp_wkernels* kern, int64_t V, const GridWork& w, const float2* grid,
               float2* vis_out, cudaStream_t st) {
    WP_CUDA(cudaMemsetAsync(vis_out, 0, sizeof(float2) * (size_t)V, st));
    if (V == 0) return WP_OK;
    int64_t threads = V * 32;
    unsigned blocks = (unsigned)((threads + 255) / 256);
    k_degrid<<<blocks, 256, 0, st>>>(g.N, g.os, g.s_max, (int)w.nbins, w.seff, kern->offsets,
                                     reinterpret_cast<const float2*>(kern->cache), w.count, w.srec, grid,
                                     vis_out, V);
    WP_LAUNCH_CHECK("k_degrid");
    return WP_OK;
}

}  // namespace wp
