// One work item of the row-owned shared-tile gridder (grid_method 3), shared by the per-call
// kernel (k_grid_ro) and the persistent multi-job kernel (k_grid_batch): item = (plane, T x T
// output tile).  The block decodes the candidates -- visibilities of the plane in the bins
// within footprint reach of the tile -- one per thread into a compact list of those whose
// footprint meets the tile (intersection rectangle, first tap, weighted value, conjugation
// flag); warp w then updates only tile rows w, w + GRID_WARPS, ..., its lanes across the
// intersection's columns, so the accumulation is a plain shared-memory read-modify-write; the
// tile is flushed to the grid once (one float2 reduction per touched cell) and cleared.
// COHERENT: the binned records were written by the same launch (read through L2, not the
// non-coherent read-only path).
#pragma once

#include "wp_internal.cuh"

namespace wp {

constexpr int GRID_WARPS = 8;              // warps per gridding block
constexpr int RO_LIST = GRID_WARPS * 32;   // candidates decoded per round (one per thread)

template <bool COHERENT>
__device__ __forceinline__ int4 ld_rec(const int4* p) { return COHERENT ? __ldcg(p) : __ldg(p); }
template <bool COHERENT>
__device__ __forceinline__ float2 ld_vis(const float2* p) { return COHERENT ? __ldcg(p) : __ldg(p); }

template <int TILE, bool COHERENT>
__device__ __forceinline__ void ro_item(int item, int N, int os, int s_max, int ntx, int ntiles,
                                        const int32_t* __restrict__ support, const int64_t* __restrict__ offsets,
                                        const float2* __restrict__ cache, const int* __restrict__ start,
                                        const int4* __restrict__ srec, const float2* __restrict__ svis,
                                        float2* __restrict__ grid, float2* tile, int* l_off, uint32_t* l_geo,
                                        float2* l_vv, int* s_n_ptr) {
    constexpr int CH = TILE / 32;                 // column chunks of a tile row
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int& s_n = *s_n_ptr;
    const int p = item / ntiles;
    const int t = item - p * ntiles;
    const int oy = t / ntx, ox = t - oy * ntx;
    const int S = min(max(support[p], 1), s_max);
    const int W = 2 * S + 1;
    const int W2 = W * W;
    const int D = (S + TILE - 1) / TILE;
    const float2* pcache = cache + offsets[p];
    const int64_t blk = offsets[p + 1] - offsets[p];   // the plane's block (checked build)
    const int ty0 = oy * TILE, tx0 = ox * TILE;
    const int cx_lo = max(0, ox - D), cx_hi = min(ntx - 1, ox + D);
    for (int cy = max(0, oy - D); cy <= min(ntx - 1, oy + D); ++cy) {
        const int kb = p * ntiles + cy * ntx;
        const int beg = start[kb + cx_lo], end = start[kb + cx_hi + 1];
        for (int base = beg; base < end; base += RO_LIST) {
            // decode: one candidate per thread, compacted into the list
            if (threadIdx.x == 0) s_n = 0;
            __syncthreads();
            const int q = base + (int)threadIdx.x;
            if (q < end) {
                const int4 r4 = ld_rec<COHERENT>(srec + q);
                const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
                const int c0 = max(iu - S, tx0), c1 = min(iu + S, tx0 + TILE - 1);
                const int r0 = max(iv - S, ty0), r1 = min(iv + S, ty0 + TILE - 1);
                if (c0 <= c1 && r0 <= r1) {
                    // per-thread slots: the list order scatters runs of neighbouring
                    // visibilities (same baseline, consecutive dumps), whose identical
                    // rectangles would otherwise chain each warp's shared-memory updates
                    const int slot = atomicAdd(&s_n, 1);
                    const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
                    l_off[slot] = (fv * os + fu) * W2 + (r0 - (iv - S)) * W + (c0 - (iu - S));
                    l_geo[slot] = (uint32_t)(r0 - ty0) | ((uint32_t)(r1 - ty0) << 8) |
                                  ((uint32_t)(c0 - tx0) << 16) | ((uint32_t)(c1 - c0) << 24) |
                                  ((uint32_t)((r4.y >> 16) & 1) << 31);
                    l_vv[slot] = ld_vis<COHERENT>(svis + q);
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
                const float2* sub = pcache + l_off[e] + (rw - r0) * W;
                int64_t tix = (int64_t)l_off[e] + (int64_t)(rw - r0) * W;   // element of sub (checked build)
                float2* trow = tile + rw * TILE + c0;
                for (int r = rw; r <= r1; r += GRID_WARPS) {
                    float2 tp[CH];
#pragma unroll
                    for (int k = 0; k < CH; ++k)
                        tp[k] = (lane + 32 * k < w && in_bounds(tix + lane + 32 * k, blk, BS_TAP))
                                    ? __ldg(sub + lane + 32 * k) : make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int k = 0; k < CH; ++k) {
                        if (lane + 32 * k < w) {
                            const float ti = sgn * tp[k].y;
                            float2 a = trow[lane + 32 * k];
                            a.x = fmaf(vv.x, tp[k].x, fmaf(-vv.y, ti, a.x));
                            a.y = fmaf(vv.x, ti, fmaf(vv.y, tp[k].x, a.y));
                            trow[lane + 32 * k] = a;
                        }
                    }
                    sub += GRID_WARPS * W;
                    tix += GRID_WARPS * W;
                    trow += GRID_WARPS * TILE;
                }
                __syncwarp();   // the next entry may touch this one's cells from other lanes
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
            if (gy < N && gx < N && in_bounds((int64_t)gy * N + gx, (int64_t)N * N, BS_GRID))
                atomicAdd(grid + (int64_t)gy * N + gx, a);
            tile[i] = make_float2(0.0f, 0.0f);
        }
    }
    __syncthreads();
}

}  // namespace wp
