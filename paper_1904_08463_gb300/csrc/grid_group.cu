// Gridding over groups of planes (grid_method 5 and 6; Alg. 1 / Alg. 2 gridding step).
//
// The per-plane gridders flush each (plane, output tile) item to the grid with one float2
// reduction per touched cell, so every grid cell is reduced into once per plane whose
// footprints reach it.  On the full-imaging workload (8M visibilities, 512 planes, 4096^2) the
// union of a plane's footprints is 3.9 % of its taps: 2.1 G global reductions per call, which
// at the measured rate of random float2 reductions over a 128 MB grid (~80 G/s) is a large
// part of the gridding time.  Neighbouring |w| planes come from the same baselines at nearby
// hour angles, so their footprints cover nearly the same cells: an item that owns one output
// tile for a group of GG_PLANES consecutive planes accumulates all of them before its single
// flush, and the union over a group of 8 is 0.7 % of the taps (0.29 G reductions).
//
// Work item = (plane group, T x T output tile), live when a visibility of one of the group's
// planes sits within footprint reach of the tile.  Per item the block lists the bins of every
// plane of the group within reach (segments of the uv-sorted records), decodes the candidates
// in rounds of one per thread into a compact list of those whose footprint meets the tile
// (first tap of the intersection, row stride, rectangle, complex coefficients with the
// conjugation of w < 0 folded in), then accumulates:
//   method 5  into a shared-memory tile, warp w owning rows w, w + 8, ..., lanes across the
//             intersection's columns (a plain read-modify-write: no two lanes or warps share a
//             cell), flushed once per item;
//   method 6  into registers, warp w holding its rows w + 8 i, lane l columns l + 32 k, each
//             (row, entry) pair visited row by row, flushed from registers once per item.
#include <cuda_runtime.h>

#include "wp_internal.cuh"

namespace wp {

namespace {
constexpr int GG_WARPS = 8;
constexpr int GG_LIST = GG_WARPS * 32;          // candidates decoded per round (one per thread)
constexpr int GG_PLANES = 8;                    // planes per group
constexpr int GG_MAX_ROWS = 2 * ((511 + 31) / 32) + 1;   // bin rows within reach, T >= 32, S <= 511
constexpr int GG_MAXSEG = GG_PLANES * GG_MAX_ROWS;
}  // namespace

int grid_group_planes() { return GG_PLANES; }

// Work-item flags of the grouped gridders: (group, tile) is live if any plane of the group has a
// visibility within its footprint reach (ceil(S_p / T) tiles) of the tile.
__global__ void __launch_bounds__(256) k_item_flags_group(int P, int ngrp, int T, int ntx, int ntiles, int s_max,
                                                          const int32_t* __restrict__ support,
                                                          const int* __restrict__ start, int* __restrict__ flags) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)ngrp * ntiles;
    if (it >= n) return;
    const int grp = (int)(it / ntiles);
    const int t = (int)(it - (int64_t)grp * ntiles);
    const int oy = t / ntx, ox = t - oy * ntx;
    int any = 0;
    for (int p = grp * GG_PLANES; p < min(P, (grp + 1) * GG_PLANES) && !any; ++p) {
        const int D = (min(max(support[p], 1), s_max) + T - 1) / T;
        const int* s = start + (int64_t)p * ntiles;
        const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
        for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy)
            any |= (s[cy * ntx + cx_hi + 1] > s[cy * ntx + cx_lo]);
    }
    flags[it] = any;
}

template <int TILE, bool REG>
__global__ void __launch_bounds__(GG_WARPS * 32) k_grid_grp(int N, int os, int s_max, int P, int ntx, int ntiles,
                                                            const int32_t* __restrict__ support,
                                                            const int64_t* __restrict__ offsets,
                                                            const float2* __restrict__ cache,
                                                            const int* __restrict__ start,
                                                            const int4* __restrict__ srec,
                                                            const float2* __restrict__ svis,
                                                            const int* __restrict__ items,
                                                            int* __restrict__ ctrl, float2* __restrict__ grid) {
    constexpr int CH = TILE / 32;                 // column chunks of a tile row
    constexpr int RPW = TILE / GG_WARPS;          // rows per warp
    __shared__ float2 tile[REG ? 1 : TILE * TILE];
    __shared__ long long l_off[GG_LIST];          // element offset of the intersection's first tap
    __shared__ uint32_t l_geo[GG_LIST];           // r0 | r1 << 8 | c0 << 16 | (w - 1) << 24
    __shared__ int l_w[GG_LIST];                  // row stride (2S + 1) of the entry's plane
    __shared__ float4 l_cf[GG_LIST];              // (Re V, -s Im V, s Re V, Im V), s = -1 for w < 0
    __shared__ int seg_beg[GG_MAXSEG];
    __shared__ int seg_pre[GG_MAXSEG + 1];
    __shared__ int s_item, s_n, s_nseg;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n_items = ctrl[1];
    float2 acc[REG ? RPW : 1][CH];
    if (!REG)
        for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) tile[i] = make_float2(0.0f, 0.0f);
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
        const int ty0 = oy * TILE, tx0 = ox * TILE;
        // ---- segments: the bin rows within reach of the tile, for every plane of the group
        if (wid == 0) {
            const int p = grp * GG_PLANES + lane;
            int rows = 0, cy_lo = 0, cx_lo = 0, cx_hi = 0;
            if (lane < GG_PLANES && p < P) {
                const int D = (min(max(support[p], 1), s_max) + TILE - 1) / TILE;
                cy_lo = max(0, oy - D);
                rows = min(ntx - 1, oy + D) - cy_lo + 1;
                cx_lo = max(0, ox - D);
                cx_hi = min(ntx - 1, ox + D);
            }
            int pre = rows;                       // inclusive scan over the lanes
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += v;
            }
            const int base = pre - rows;
            for (int r = 0; r < rows; ++r) {
                const int kb = p * ntiles + (cy_lo + r) * ntx;
                const int beg = start[kb + cx_lo];
                seg_beg[base + r] = beg;
                seg_pre[base + r + 1] = start[kb + cx_hi + 1] - beg;   // length, scanned below
            }
            const int nseg = __shfl_sync(0xffffffffu, pre, 31);
            __syncwarp();
            // exclusive prefix of the lengths, 32 at a time
            int carry = 0;
            if (lane == 0) seg_pre[0] = 0;
            for (int b = 0; b < nseg; b += 32) {
                int v = (b + lane < nseg) ? seg_pre[b + lane + 1] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += u;
                }
                if (b + lane < nseg) seg_pre[b + lane + 1] = carry + v;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
            if (lane == 0) s_nseg = nseg;
        }
        if (REG) {
#pragma unroll
            for (int i = 0; i < RPW; ++i)
#pragma unroll
                for (int k = 0; k < CH; ++k) acc[i][k] = make_float2(0.0f, 0.0f);
        }
        __syncthreads();
        const int nseg = s_nseg;
        const int ntot = seg_pre[nseg];
        for (int base = 0; base < ntot; base += GG_LIST) {
            // ---- decode one candidate per thread into the compact list
            if (threadIdx.x == 0) s_n = 0;
            __syncthreads();
            const int c = base + (int)threadIdx.x;
            if (c < ntot) {
                int lo = 0, hi = nseg;                 // largest s with seg_pre[s] <= c
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (seg_pre[mid] <= c) lo = mid; else hi = mid;
                }
                const int q = seg_beg[lo] + (c - seg_pre[lo]);
                const int4 r4 = __ldg(srec + q);
                const int p = r4.z;
                const int S = min(max(support[p], 1), s_max);
                const int W = 2 * S + 1;
                const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
                const int c0 = max(iu - S, tx0), c1 = min(iu + S, tx0 + TILE - 1);
                const int r0 = max(iv - S, ty0), r1 = min(iv + S, ty0 + TILE - 1);
                if (c0 <= c1 && r0 <= r1) {
                    const int slot = atomicAdd(&s_n, 1);
                    const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
                    const float sg = ((r4.y >> 16) & 1) ? -1.0f : 1.0f;
                    const float2 vv = __ldg(svis + q);
                    l_off[slot] = offsets[p] + (long long)(fv * os + fu) * W * W +
                                  (long long)(r0 - (iv - S)) * W + (c0 - (iu - S));
                    l_w[slot] = W;
                    l_geo[slot] = (uint32_t)(r0 - ty0) | ((uint32_t)(r1 - ty0) << 8) |
                                  ((uint32_t)(c0 - tx0) << 16) | ((uint32_t)(c1 - c0) << 24);
                    l_cf[slot] = make_float4(vv.x, -sg * vv.y, sg * vv.x, vv.y);
                }
            }
            __syncthreads();
            const int n = s_n;
            if (!REG) {
                for (int e = 0; e < n; ++e) {
                    const uint32_t geo = l_geo[e];
                    const int r0 = (int)(geo & 0xff), r1 = (int)((geo >> 8) & 0xff);
                    const int rw = r0 + ((wid - r0) & (GG_WARPS - 1));   // first owned row
                    if (rw > r1) continue;
                    const int c0 = (int)((geo >> 16) & 0xff), w = (int)(geo >> 24) + 1;
                    const int W = l_w[e];
                    const float4 cf = l_cf[e];
                    const float2* sub = cache + l_off[e] + (long long)(rw - r0) * W;
                    float2* trow = tile + rw * TILE + c0;
                    for (int r = rw; r <= r1; r += GG_WARPS) {
                        float2 tp[CH];
#pragma unroll
                        for (int k = 0; k < CH; ++k)
                            tp[k] = (lane + 32 * k < w) ? __ldg(sub + lane + 32 * k) : make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            if (lane + 32 * k < w) {
                                float2 a = trow[lane + 32 * k];
                                a.x = fmaf(cf.x, tp[k].x, fmaf(cf.y, tp[k].y, a.x));
                                a.y = fmaf(cf.z, tp[k].y, fmaf(cf.w, tp[k].x, a.y));
                                trow[lane + 32 * k] = a;
                            }
                        }
                        sub += GG_WARPS * W;
                        trow += GG_WARPS * TILE;
                    }
                    __syncwarp();   // the next entry may touch this one's cells from other lanes
                }
            } else {
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    const int r = wid + GG_WARPS * i;
                    for (int e = 0; e < n; ++e) {
                        const uint32_t geo = l_geo[e];
                        const int r0 = (int)(geo & 0xff), r1 = (int)((geo >> 8) & 0xff);
                        if (r < r0 || r > r1) continue;
                        const int c0 = (int)((geo >> 16) & 0xff), w = (int)(geo >> 24) + 1;
                        const float2* row = cache + l_off[e] + (long long)(r - r0) * l_w[e];
                        const float4 cf = l_cf[e];
#pragma unroll
                        for (int k = 0; k < CH; ++k) {
                            const int d = lane + 32 * k - c0;
                            const float2 tp = ((unsigned)d < (unsigned)w) ? __ldg(row + d) : make_float2(0.0f, 0.0f);
                            acc[i][k].x = fmaf(cf.x, tp.x, fmaf(cf.y, tp.y, acc[i][k].x));
                            acc[i][k].y = fmaf(cf.z, tp.y, fmaf(cf.w, tp.x, acc[i][k].y));
                        }
                    }
                }
            }
            __syncthreads();   // the list is rebuilt for the next round
        }
        // ---- flush the tile once per item (one float2 reduction per touched cell)
        if (!REG) {
            for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
                const float2 a = tile[i];
                if (a.x != 0.0f || a.y != 0.0f) {
                    const int gy = ty0 + i / TILE, gx = tx0 + (i & (TILE - 1));
                    if (gy < N && gx < N) atomicAdd(grid + (int64_t)gy * N + gx, a);
                    tile[i] = make_float2(0.0f, 0.0f);
                }
            }
            __syncthreads();
        } else {
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                const int gy = ty0 + wid + GG_WARPS * i;
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const int gx = tx0 + lane + 32 * k;
                    if ((acc[i][k].x != 0.0f || acc[i][k].y != 0.0f) && gy < N && gx < N)
                        atomicAdd(grid + (int64_t)gy * N + gx, acc[i][k]);
                }
            }
        }
    }
}

// Items, then the grouped gridder (grid_method 5: shared tile; 6: row registers).
int grid_run_group(const Geom& g, const wp_wkernels* kern, const GridWork& w, float2* grid, cudaStream_t st) {
    const int P = kern->P;
    const int ngrp = (P + GG_PLANES - 1) / GG_PLANES;
    const int64_t n = (int64_t)ngrp * w.ntiles;
    k_item_flags_group<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, ngrp, w.T, w.ntx, w.ntiles, g.s_max, w.seff,
                                                                    w.count, w.flags);
    WP_LAUNCH_CHECK("k_item_flags_group");
    int rc = exclusive_scan_i32(w.flags, w.cursor, n, w.scan_tmp, st);
    if (rc) return rc;
    rc = write_items(n, w, st);
    if (rc) return rc;
    int dev = 0, sms = 0, per_sm = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const float2* c2 = reinterpret_cast<const float2*>(kern->cache);
#define WP_LAUNCH_GRP(T, R)                                                                                      \
    do {                                                                                                         \
        WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_grp<T, R>, GG_WARPS * 32, 0));    \
        if (per_sm < 1) per_sm = 1;                                                                              \
        k_grid_grp<T, R><<<sms * per_sm, GG_WARPS * 32, 0, st>>>(g.N, g.os, g.s_max, P, w.ntx, w.ntiles, w.seff, \
                                                                 kern->offsets, c2, w.count, w.srec, w.svis,     \
                                                                 w.items, w.ctrl, grid);                         \
    } while (0)
    const bool reg = (g.grid_method == 6);
    if (w.T == 32) {
        if (reg) WP_LAUNCH_GRP(32, true); else WP_LAUNCH_GRP(32, false);
    } else {
        if (reg) WP_LAUNCH_GRP(64, true); else WP_LAUNCH_GRP(64, false);
    }
#undef WP_LAUNCH_GRP
    WP_LAUNCH_CHECK("k_grid_grp");
    return WP_OK;
}

}  // namespace wp
