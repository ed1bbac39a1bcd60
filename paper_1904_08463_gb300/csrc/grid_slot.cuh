// One work item of the slot gridder (grid_method 9), shared by the per-call kernel
// (k_grid_slot) and the persistent multi-job kernel (k_grid_batch): item `it` of the call's
// item list = (plane, chunk of up to SLOT_CHUNK Morton-sorted visibilities, tile of the W x W
// slots: 32 x ROWS, or 16 x 2 ROWS for the last W mod 32 <= 16 columns), processed by one warp.
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

constexpr int SLOT_ROWS = 10;        // slot rows per lane of the gridder (registers: sum, cell offset each)
constexpr int SLOT_DEGRID_ROWS = 8;  // slot rows per lane of the degridder
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

// a grid cell written or read by a slot (bounds-checked in the checked build)
__device__ __forceinline__ void slot_add(float2* grid, int N, int cy, int cx, float2 v) {
    if (in_bounds(cx, N, BS_GRID) && in_bounds(cy, N, BS_GRID)) atomicAdd(grid + (int64_t)cy * N + cx, v);
}
__device__ __forceinline__ float2 slot_get(const float2* grid, int N, int cy, int cx) {
    return (in_bounds(cx, N, BS_GRID) && in_bounds(cy, N, BS_GRID)) ? __ldg(grid + (int64_t)cy * N + cx)
                                                                    : make_float2(0.0f, 0.0f);
}

// a running sum worth writing (either part non-zero; -0 counts as zero)
__device__ __forceinline__ bool slot_nonzero(float2 a) {
    return ((__float_as_uint(a.x) | __float_as_uint(a.y)) & 0x7fffffffu) != 0u;
}

// Places the slots for the footprint of record r (corner x0 | y0 << 16 in r.x, the corner mod W
// in r.y): the lane's column cell cx, the cell row cyt of tile row `lane` (lanes below the
// tile's row count), every tap offset, and the sums zeroed (gridding) or the cells' grid values
// read (DEGRID).  The lane's own rows are tile rows rbase .. rbase + ROWS - 1.
template <int ROWS, bool DEGRID>
__device__ __forceinline__ void slot_place(int4 r, int W, int N, int a_res, int b_res, int nval, int rbase,
                                           const float2* __restrict__ grid, int& cx, int& cyt, unsigned& cb, unsigned (&coff)[ROWS],
                                           float2 (&acc)[ROWS]) {
    const int x0 = r.x & 0xffff, y0 = (r.x >> 16) & 0xffff;
    const int xm = r.y & 0xffff, ym = (r.y >> 16) & 0xffff;
    int nx = a_res - xm;
    nx += (nx < 0) ? W : 0;
    int ny = b_res - ym;
    ny += (ny < 0) ? W : 0;
    cx = x0 + nx;
    cyt = y0 + ny;
    cb = (unsigned)(y0 * W + x0) * 8u;
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        const int cyj = __shfl_sync(0xffffffffu, cyt, rbase + j);
        coff[j] = (unsigned)(cyj * W + cx) * 8u;
        acc[j] = (DEGRID && j < nval) ? slot_get(grid, N, cyj, cx) : make_float2(0.0f, 0.0f);
    }
}

// The plane of item `it`: the largest p with istart[p] <= it.
__device__ __forceinline__ int slot_plane(int it, int P, const int* __restrict__ istart) {
    int lo = 0, hi = P;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (istart[mid] <= it) lo = mid; else hi = mid;
    }
    return lo;
}

// Slot tiles per chunk of a plane with footprint width W: the floor(W / 32) full columns of
// 32 x ROWS tiles, and the remaining c = W mod 32 columns (if any) in 16 x 2 ROWS tiles when
// c <= 16 -- two row groups of 16 lanes, half the idle lanes of a 32-wide tile -- else in
// 32 x ROWS tiles.
__host__ __device__ __forceinline__ int slot_tiles_mixed(int W, int rows) {
    const int nys = (W + rows - 1) / rows, nf = W / 32, c = W - 32 * nf;
    const int nrem = (c == 0) ? 0 : ((c <= 16) ? (W + 2 * rows - 1) / (2 * rows) : nys);
    return nf * nys + nrem;
}

// DEGRID = false: gridding (each slot sums V x tap into its cell and flushes the sum to `grid`
// when the cell changes).  DEGRID = true: degridding, the adjoint (each slot holds the value of
// `grid` at its cell, reloaded when the cell changes; per visibility the warp sums conj(tap) x
// value over its slots and adds the sum into vis_out[original index]; svis is not read).
// One tile: plane p (width W), chunk `chunk` of its sorted visibilities, slot columns
// txs COLS .. + COLS - 1 and rows tys TR .. + TR - 1.  PREFETCH: the chunk's records are
// prefetched into L2 first (the persistent batch, whose records may have left L2 since they
// were sorted; a per-call walk runs right after its own sort and gather).
template <int ROWS, bool COHERENT, bool DEGRID, int COLS, bool PREFETCH = false>
__device__ __forceinline__ void slot_walk_tile(int p, int W, int chunk, int txs, int tys, int N,
                                               const int64_t* __restrict__ offsets, const float2* __restrict__ cache,
                                               const int* __restrict__ vstart, const int4* __restrict__ srec,
                                               const float2* __restrict__ svis, float2* __restrict__ grid,
                                               float2* __restrict__ vis_out, int64_t n_vis) {
    const int lane = threadIdx.x & 31;
    constexpr int TR = (32 / COLS) * ROWS;   // slot rows of a warp tile (one or two row groups)
    static_assert(COLS == 32 || COLS == 16, "a warp tile is 32 or 16 columns wide");
    static_assert(TR <= 32, "one lane per tile row");
    const int v0 = vstart[p] + chunk * SLOT_CHUNK;
    const int v1 = min(v0 + SLOT_CHUNK, vstart[p + 1]);
    if (v0 >= v1) return;   // no visibility (a safety net: item lists count whole chunks)
    if (PREFETCH) {
        // the chunk's records and values into L2 ahead of the walk (one prefetch per 128-byte
        // line): the walk's own loads run only one record ahead
        const char* r0 = reinterpret_cast<const char*>(srec + v0);
        const int rb = (v1 - v0) * (int)sizeof(int4);
        for (int o = lane * 128; o < rb; o += 32 * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(r0 + o));
        if (!DEGRID) {
            const char* s0 = reinterpret_cast<const char*>(svis + v0);
            const int sb = (v1 - v0) * (int)sizeof(float2);
            for (int o = lane * 128; o < sb; o += 32 * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(s0 + o));
        }
    }
    const float2* pc = cache + offsets[p];
    const int64_t blk = offsets[p + 1] - offsets[p];   // the plane's block (checked build)
    const int a = txs * COLS + lane % COLS;   // the lane's slot column
    const bool a_ok = a < W;
    const int b0 = tys * TR;                  // slot rows b0 .. b0 + TR - 1 of the tile
    const int rbase = (lane / COLS) * ROWS;   // the lane's rows: b0 + rbase .. b0 + rbase + ROWS - 1
    const int nrows = max(0, min(ROWS, W - b0 - rbase));   // of them inside the W x W residues
    // Slot (lane, j) sums the cell (cx, cy[j]): column cx of the lane, row cy[j] of row j.  Its
    // tap in the footprint with corner (x0, y0) is (cx - x0, cy[j] - y0), at byte offset
    // ((cy[j] - y0) W + cx - x0) x 8 = coff[j] - cb of the sub-kernel, coff[j] = (cy[j] W + cx) x 8
    // depending on the cell alone and cb = (y0 W + x0) x 8 on the corner alone.  A footprint move
    // keeps every cell and changes cb only; a slot whose cell leaves the new footprint (cx - x0
    // or cy[j] - y0 outside [0, W)) writes its sum to the grid and moves its cell by a period W.  The row
    // cells are the same in every lane of a row group and live one per lane (lane k < TR holds
    // the cell row of tile row k), so the rows that move are one ballot and the columns that move
    // one vote.  Lanes and rows beyond
    // the W x W residues track the residue a mod W (b mod W) of a slot that exists, so every tap
    // offset stays inside the sub-kernel; they are never flushed.  (For DEGRID, acc[j] holds the
    // grid value at the slot's cell instead of a running sum, reloaded when the cell moves.)
    const unsigned FULL = 0xffffffffu;
    const int a_res = a % W;
    const int b_res = (b0 + (lane < TR ? lane : 0)) % W;
    const int nval = a_ok ? nrows : 0;        // rows j < nval of this lane are real slots
    float2 acc[ROWS];
    unsigned coff[ROWS];                      // (cy[j] W + cx) x 8: the cell's part of the tap offset
    unsigned cb;                              // (y0 W + x0) x 8 of the current corner
    int4 rn = ld_slot_rec<COHERENT>(srec + v0);
    float2 vn = DEGRID ? make_float2(0.0f, 0.0f) : ld_slot_vis<COHERENT>(svis + v0);
    uint32_t prev = (uint32_t)rn.x;           // corner of the current footprint: x0 | y0 << 16
    int cx, cyt;
    slot_place<ROWS, DEGRID>(rn, W, N, a_res, b_res, nval, rbase, grid, cx, cyt, cb, coff, acc);
    for (int q = v0; q < v1; ++q) {
        const int4 r = rn;
        const float2 v = vn;
        if (q + 1 < v1) {                     // the next record while this one's taps load
            rn = ld_slot_rec<COHERENT>(srec + q + 1);
            if (!DEGRID) vn = ld_slot_vis<COHERENT>(svis + q + 1);
        }
        if ((uint32_t)r.x != prev) {          // the footprint moved
            const int x0 = r.x & 0xffff, y0 = (r.x >> 16) & 0xffff;
            const int dx = x0 - (int)(prev & 0xffffu), dy = y0 - (int)(prev >> 16);
            prev = (uint32_t)r.x;
            if (dx >= W || dx <= -W || dy >= W || dy <= -W) {
                // a long jump: every slot writes its sum and is placed anew
                if (!DEGRID) {
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        const int cyj = __shfl_sync(FULL, cyt, rbase + j);
                        const float2 sj = acc[j];
                        if (j < nval && slot_nonzero(sj)) slot_add(grid, N, cyj, cx, sj);
                    }
                }
                slot_place<ROWS, DEGRID>(r, W, N, a_res, b_res, nval, rbase, grid, cx, cyt, cb, coff, acc);
            } else {
                cb = (unsigned)(y0 * W + x0) * 8u;
                int tx = cx - x0;                 // the lane's column moves when tx leaves [0, W)
                const bool xw = (unsigned)tx >= (unsigned)W;
                const unsigned rm = __ballot_sync(FULL, lane < TR && (unsigned)(cyt - y0) >= (unsigned)W);
                const unsigned my_rm = rm >> rbase;   // bit j: the lane's row j moves
                if (__any_sync(FULL, xw)) {       // columns that move: every row of those lanes
                    tx += (tx < 0) ? W : ((tx >= W) ? -W : 0);
                    const int cxn = x0 + tx;
                    const unsigned dxo = (unsigned)(cxn - cx) * 8u;
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        const int cyj = __shfl_sync(FULL, cyt, rbase + j);
                        if (!DEGRID) {
                            const float2 sj = acc[j];
                            if (xw && j < nval && slot_nonzero(sj)) slot_add(grid, N, cyj, cx, sj);
                            acc[j] = xw ? make_float2(0.0f, 0.0f) : acc[j];
                        }
                        coff[j] += xw ? dxo : 0u;
                    }
                    cx = cxn;
                }
                if (rm) {                            // rows that move: every lane of those rows
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        // row j of some row group moves (the same test in every lane)
                        const bool any_j = (COLS == 32) ? ((rm >> j) & 1u) : (((rm >> j) | (rm >> (ROWS + j))) & 1u);
                        if (any_j) {
                            const int cyj = __shfl_sync(FULL, cyt, rbase + j);
                            if ((my_rm >> j) & 1u) {
                                const int cyn = cyj + ((cyj < y0) ? W : -W);
                                if (!DEGRID) {
                                    const float2 sj = acc[j];
                                    if (j < nval && slot_nonzero(sj)) slot_add(grid, N, cyj, cx, sj);
                                    acc[j] = make_float2(0.0f, 0.0f);
                                }
                                coff[j] += (unsigned)((cyn - cyj) * W) * 8u;
                                if (DEGRID && j < nval) acc[j] = slot_get(grid, N, cyn, cx);
                            }
                        }
                    }
                    if (lane < TR && ((rm >> lane) & 1u)) cyt += (cyt < y0) ? W : -W;
                }
                if (DEGRID && __any_sync(FULL, xw)) {    // moved columns read their new cells
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        const int cyj = __shfl_sync(FULL, cyt, rbase + j);
                        if (xw && j < nval) acc[j] = slot_get(grid, N, cyj, cx);
                    }
                }
            }
        }
        // tap (cx - x0, cy[j] - y0) of the sub-kernel: byte offset coff[j] - cb from its start
        const char* sub = reinterpret_cast<const char*>(pc + (r.z & 0x7fffffff)) - (int64_t)cb;
        const float sg = (r.z < 0) ? -1.0f : 1.0f;
        float2 tp[ROWS];
#pragma unroll
        for (int j = 0; j < ROWS; ++j)
            tp[j] = in_bounds((int64_t)(r.z & 0x7fffffff) + ((int64_t)coff[j] - (int64_t)cb) / 8, blk, BS_TAP)
                        ? __ldg(reinterpret_cast<const float2*>(sub + coff[j])) : make_float2(0.0f, 0.0f);
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
            if (lane == 0 && (sr != 0.0f || si != 0.0f) && in_bounds(r.w, n_vis, BS_VIS))
                atomicAdd(vis_out + r.w, make_float2(sr, si));
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
        for (int j = 0; j < ROWS; ++j) {
            const int cyj = __shfl_sync(FULL, cyt, rbase + j);
            const float2 sj = acc[j];
            if (j < nval && slot_nonzero(sj)) slot_add(grid, N, cyj, cx, sj);
        }
    }
}

// Item `it` of an item list of slot_tiles_mixed tiles per chunk: the gridder (per call and in
// the persistent batch) and, with DEGRID, the slot degridder.
template <int ROWS, bool COHERENT, bool DEGRID = false, bool PREFETCH = false>
__device__ __forceinline__ void slot_item(int it, int N, int P, int s_max, const int32_t* __restrict__ support,
                                          const int64_t* __restrict__ offsets, const float2* __restrict__ cache,
                                          const int* __restrict__ vstart, const int* __restrict__ istart,
                                          const int4* __restrict__ srec, const float2* __restrict__ svis,
                                          float2* __restrict__ grid, float2* __restrict__ vis_out = nullptr,
                                          int64_t n_vis = 0) {
    const int p = slot_plane(it, P, istart);
    const int W = 2 * min(max(support[p], 1), s_max) + 1;
    const int nys = (W + ROWS - 1) / ROWS, nf = W / 32, c = W - 32 * nf;
    const int T = slot_tiles_mixed(W, ROWS);
    const int local = it - istart[p];
    const int chunk = local / T;
    const int tt = local - chunk * T;
    if (tt < nf * nys) {                      // a full 32-column tile
        const int tys = tt / nf;
        slot_walk_tile<ROWS, COHERENT, DEGRID, 32, PREFETCH>(p, W, chunk, tt - tys * nf, tys, N, offsets, cache, vstart, srec,
                                                   svis, grid, vis_out, n_vis);
    } else if (c <= 16) {                     // the remaining columns, 16 x 2 ROWS tiles
        slot_walk_tile<ROWS, COHERENT, DEGRID, 16, PREFETCH>(p, W, chunk, 2 * nf, tt - nf * nys, N, offsets, cache, vstart,
                                                   srec, svis, grid, vis_out, n_vis);
    } else {                                  // the remaining columns, 32 x ROWS tiles
        slot_walk_tile<ROWS, COHERENT, DEGRID, 32, PREFETCH>(p, W, chunk, nf, tt - nf * nys, N, offsets, cache, vstart, srec,
                                                   svis, grid, vis_out, n_vis);
    }
}

}  // namespace wp
