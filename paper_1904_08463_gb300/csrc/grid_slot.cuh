// One work item of the slot gridder (grid_method 9), shared by the per-call kernel
// (k_grid_slot) and the persistent multi-job kernel (k_grid_batch): item `it` of the call's
// item list = (plane, chunk of up to SLOT_CHUNK Morton-sorted visibilities, 32 x ROWS tile of the
// W x W slots), processed by one warp.
//
// Every tap of a (2S+1)^2 footprint whose corner is (x0, y0) lands on a distinct residue class
// (x mod W, y mod W), W = 2S+1.  The lane owning the residue (a, b) -- a "slot" -- therefore has
// exactly one tap of every visibility of the plane: the cell x = x0 + ((a - x0) mod W) (same for
// y), tap offset (x - x0, y - y0).  It keeps that cell's sum in a register and writes it to the
// grid (one float2 reduction) only when a later visibility moves its cell.  Slots outside the
// W x W residues (lane columns a >= W of the last column tile, rows b >= W of the last row tile)
// read tap 0 of the sub-kernel -- always in bounds -- and are never flushed, so the tap loads
// need no guard.  COHERENT: the sorted records were written by the same launch (read through
// L2, not the non-coherent read-only path).
#pragma once

#include "wp_internal.cuh"

namespace wp {

constexpr int SLOT_ROWS = 10;        // slot rows per lane (registers: sum, tap row, tap offset each)
constexpr int SLOT_CHUNK = 512;      // visibilities per work item
constexpr int SLOT_WARPS = 8;        // warps per block

template <bool COHERENT>
__device__ __forceinline__ int4 ld_slot_rec(const int4* p) { return COHERENT ? __ldcg(p) : __ldg(p); }
template <bool COHERENT>
__device__ __forceinline__ float2 ld_slot_vis(const float2* p) { return COHERENT ? __ldcg(p) : __ldg(p); }

// Sorted record i of the slot gridder: x = x0 | y0 << 16 (footprint corner), y = (x0 mod W) |
// (y0 mod W) << 16, z = sub-kernel offset (fv os + fu) W^2 | conj << 31, w = original index; the
// weighted value beside it.  idx: the sort's permutation; rec: the unsorted binning records.
__device__ __forceinline__ void slot_gather_one(int64_t i, int os, int s_max, const uint32_t* __restrict__ idx,
                                                const int4* __restrict__ rec, const int32_t* __restrict__ support,
                                                const float2* __restrict__ vis, const float* __restrict__ weight,
                                                int4* __restrict__ srec, float2* __restrict__ svis) {
    const int k = (int)idx[i];
    const int4 r = rec[k];
    const int p = r.z;
    const int S = min(max(support[p], 1), s_max);
    const int W = 2 * S + 1;
    const int x0 = (r.x & 0xffff) - S, y0 = ((r.x >> 16) & 0xffff) - S;
    const int fu = r.y & 0xff, fv = (r.y >> 8) & 0xff, conj = (r.y >> 16) & 1;
    srec[i] = make_int4(x0 | (y0 << 16), (x0 % W) | ((y0 % W) << 16),
                        (int)((uint32_t)((fv * os + fu) * W * W) | ((uint32_t)conj << 31)), k);
    if (svis) {
        const float2 v = vis[k];
        const float a = weight ? weight[k] : 1.0f;
        svis[i] = make_float2(v.x * a, v.y * a);
    }
}

// DEGRID = false: gridding (each slot sums V x tap into its cell and flushes the sum to `grid`
// when the cell changes).  DEGRID = true: degridding, the adjoint (each slot holds the value of
// `grid` at its cell, reloaded when the cell changes; per visibility the warp sums conj(tap) x
// value over its slots and adds the sum into vis_out[original index]; svis is not read).
template <int ROWS, bool COHERENT, bool DEGRID>
__device__ __forceinline__ void slot_walk(int it, int N, int P, int s_max, const int32_t* __restrict__ support,
                                          const int64_t* __restrict__ offsets, const float2* __restrict__ cache,
                                          const int* __restrict__ vstart, const int* __restrict__ istart,
                                          const int4* __restrict__ srec, const float2* __restrict__ svis,
                                          float2* __restrict__ grid, float2* __restrict__ vis_out) {
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = P;                       // largest plane with istart <= it
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (istart[mid] <= it) lo = mid; else hi = mid;
    }
    const int p = lo;
    const int S = min(max(support[p], 1), s_max);
    const int W = 2 * S + 1;
    const int nxs = (W + 31) >> 5, nys = (W + ROWS - 1) / ROWS;
    const int local = it - istart[p];
    const int chunk = local / (nxs * nys);
    const int tt = local - chunk * (nxs * nys);
    const int tys = tt / nxs, txs = tt - tys * nxs;
    const int v0 = vstart[p] + chunk * SLOT_CHUNK;
    const int v1 = min(v0 + SLOT_CHUNK, vstart[p + 1]);
    const float2* pc = cache + offsets[p];
    const int a = txs * 32 + lane;            // the lane's slot column
    const bool a_ok = a < W;
    const int b0 = tys * ROWS;                // slot rows b0 .. b0 + ROWS - 1
    const int nrows = min(ROWS, W - b0);      // rows of this tile inside the W x W residues
    // (for DEGRID, acc[j] holds the grid value at the slot's cell instead of a running sum)
    // Slot (lane, j) has the tap (jx, jy[j]) of the current footprint and sums the cell
    // (x0 + jx, y0 + jy[j]).  A move of the footprint corner by (dx, dy), |dx|, |dy| < W, changes
    // the lane's column only if jx - dx leaves [0, W) (the cell moves by one period) and row j's
    // only if jy[j] - dy does; every other slot keeps its cell and shifts its tap offset.  Larger
    // moves recompute everything.
    // (for DEGRID, acc[j] holds the grid value at the slot's cell instead of a running sum)
    // Slot (lane, j) has the tap (jx, jy[j]) of the current footprint and sums the cell
    // (x0 + jx, y0 + jy[j]).  A move of the footprint corner by (dx, dy), |dx|, |dy| < W, changes
    // the lane's column only if jx - dx leaves [0, W) (the cell moves by one period) and row j's
    // only if jy[j] - dy does; every other slot keeps its cell and shifts its tap offset.  Larger
    // moves recompute everything.  Lanes and rows beyond the W x W residues track the residue
    // a mod W (b mod W) of a slot that exists, so that every tap offset is always inside the
    // sub-kernel; they are never flushed.
    const int a_res = a % W;
    float2 acc[ROWS];
    int jy[ROWS];
    unsigned toff[ROWS];                      // byte offset of the slot's tap in its sub-kernel
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        acc[j] = make_float2(0.0f, 0.0f);
        jy[j] = 0;
        toff[j] = 0;
    }
    int jx = 0;
    int x0p = -1, y0p = -1;                   // corner of the previous footprint (none yet)
    uint32_t prev = 0xffffffffu;              // no footprint corner packs to this
    int4 rn = ld_slot_rec<COHERENT>(srec + v0);
    float2 vn = DEGRID ? make_float2(0.0f, 0.0f) : ld_slot_vis<COHERENT>(svis + v0);
    for (int q = v0; q < v1; ++q) {
        const int4 r = rn;
        const float2 v = vn;
        if (q + 1 < v1) {                     // the next record while this one's taps load
            rn = ld_slot_rec<COHERENT>(srec + q + 1);
            if (!DEGRID) vn = ld_slot_vis<COHERENT>(svis + q + 1);
        }
        if ((uint32_t)r.x != prev) {          // the footprint moved: new cells for some slots
            prev = (uint32_t)r.x;
            const int x0 = r.x & 0xffff, y0 = (r.x >> 16) & 0xffff;
            const int dx = x0 - x0p, dy = y0 - y0p;
            if (x0p < 0 || dx >= W || dx <= -W || dy >= W || dy <= -W) {
                // first footprint or a long jump: every slot flushes (gridding) and starts over
                const int xm = r.y & 0xffff, ym = (r.y >> 16) & 0xffff;
                if (!DEGRID) {
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        if (a_ok && j < nrows && (acc[j].x != 0.0f || acc[j].y != 0.0f))
                            atomicAdd(grid + (int64_t)(y0p + jy[j]) * N + (x0p + jx), acc[j]);
                        acc[j] = make_float2(0.0f, 0.0f);
                    }
                }
                int nx = a_res - xm;
                nx += (nx < 0) ? W : 0;
                jx = nx;
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    int ny = (b0 + j) % W - ym;
                    ny += (ny < 0) ? W : 0;
                    jy[j] = ny;
                    toff[j] = (unsigned)(ny * W + nx) * 8u;
                    if (DEGRID)
                        acc[j] = (a_ok && j < nrows) ? __ldg(grid + (int64_t)(y0 + ny) * N + (x0 + nx)) : make_float2(0.0f, 0.0f);
                }
            } else if (!__any_sync(0xffffffffu, jx - dx < 0 || jx - dx >= W ||
                                                 (lane < ROWS && (jy[0] + lane >= W || jy[0] + lane - dy < 0 ||
                                                                  jy[0] + lane - dy >= W)))) {
                // no slot of this warp changes its cell: row j's tap row is jy[0] + j here (a
                // tile whose rows pass W counts as a change above), and every tap offset shifts
                // by the same amount
                const unsigned d = (unsigned)(dy * W + dx) * 8u;
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    jy[j] -= dy;
                    toff[j] -= d;
                }
                jx -= dx;
            } else {
                int nx = jx - dx;
                const bool xw = nx < 0 || nx >= W;            // the lane's column changes period
                nx += (nx < 0) ? W : ((nx >= W) ? -W : 0);
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    int ny = jy[j] - dy;
                    const bool yw = ny < 0 || ny >= W;        // row j changes period
                    ny += (ny < 0) ? W : ((ny >= W) ? -W : 0);
                    if (xw || yw) {
                        if (DEGRID) {
                            if (a_ok && j < nrows) acc[j] = __ldg(grid + (int64_t)(y0 + ny) * N + (x0 + nx));
                        } else {
                            if (a_ok && j < nrows && (acc[j].x != 0.0f || acc[j].y != 0.0f))
                                atomicAdd(grid + (int64_t)(y0p + jy[j]) * N + (x0p + jx), acc[j]);
                            acc[j] = make_float2(0.0f, 0.0f);
                        }
                    }
                    jy[j] = ny;
                    toff[j] = (unsigned)(ny * W + nx) * 8u;
                }
                jx = nx;
            }
            x0p = x0;
            y0p = y0;
        }
        const float2* sub = pc + (r.z & 0x7fffffff);
        const float sg = (r.z < 0) ? -1.0f : 1.0f;
        float2 tp[ROWS];
#pragma unroll
        for (int j = 0; j < ROWS; ++j) tp[j] = __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const char*>(sub) + toff[j]));
        if (DEGRID) {
            // conj(K) x value, K conjugated for w < 0: (tx, s ty)* (gx, gy)
            float sr = 0.0f, si = 0.0f;
#pragma unroll
            for (int j = 0; j < ROWS; ++j) {
                const float ti = sg * tp[j].y;
                sr = fmaf(tp[j].x, acc[j].x, fmaf(ti, acc[j].y, sr));
                si = fmaf(tp[j].x, acc[j].y, fmaf(-ti, acc[j].x, si));
            }
            for (int o = 16; o; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0 && (sr != 0.0f || si != 0.0f)) atomicAdd(vis_out + r.w, make_float2(sr, si));
        } else {
            const float cA = v.x, cB = -sg * v.y, cC = sg * v.x, cD = v.y;
#pragma unroll
            for (int j = 0; j < ROWS; ++j) {
                acc[j].x = fmaf(cA, tp[j].x, fmaf(cB, tp[j].y, acc[j].x));
                acc[j].y = fmaf(cC, tp[j].y, fmaf(cD, tp[j].x, acc[j].y));
            }
        }
    }
    if (!DEGRID) {
#pragma unroll
        for (int j = 0; j < ROWS; ++j)
            if (a_ok && j < nrows && (acc[j].x != 0.0f || acc[j].y != 0.0f))
                atomicAdd(grid + (int64_t)(y0p + jy[j]) * N + (x0p + jx), acc[j]);
    }
}

template <int ROWS, bool COHERENT>
__device__ __forceinline__ void slot_item(int it, int N, int P, int s_max, const int32_t* __restrict__ support,
                                          const int64_t* __restrict__ offsets, const float2* __restrict__ cache,
                                          const int* __restrict__ vstart, const int* __restrict__ istart,
                                          const int4* __restrict__ srec, const float2* __restrict__ svis,
                                          float2* __restrict__ grid) {
    slot_walk<ROWS, COHERENT, false>(it, N, P, s_max, support, offsets, cache, vstart, istart, srec, svis, grid,
                                     nullptr);
}

}  // namespace wp
