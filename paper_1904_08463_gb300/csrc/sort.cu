// Stable least-significant-digit radix sort on the device of unsigned keys (32 or 64 bit), with
// an optional uint32 value carried along, 8-bit digits, only as many passes as the keys have
// significant bits.  Used to sort the |w| of the visibilities for the plane values (Alg. 2
// steps 1-3: the bit patterns of non-negative floats order like the floats).
//
// One pass = three launches:
//   k_rs_hist     per tile of TILE keys, the digit histogram, written digit-major so that one
//                 exclusive scan over [digit][tile] gives every (digit, tile) its output base;
//   scan          exclusive_scan_i32 over 256 x n_tiles counts;
//   k_rs_scatter  per tile, each warp ranks its 256 keys among equal digits in index order
//                 (match_any + popc), warps are offset by the counts of earlier warps, and the
//                 pair is written at base + rank -- the order of equal digits is preserved, which
//                 is what makes the passes compose into a sort.
#include <cuda_runtime.h>

#include "wp_internal.cuh"

namespace wp {
namespace {
constexpr int RS_WARPS = 8;
constexpr int RS_ITEMS = 8;                                // keys per lane
constexpr int RS_WARP_KEYS = 32 * RS_ITEMS;                // 256, a warp's contiguous sub-tile
constexpr int RS_TILE = RS_WARPS * RS_WARP_KEYS;           // 2048 keys per block

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
}  // namespace

template <class KT>
__global__ void __launch_bounds__(RS_WARPS * 32) k_rs_hist(const KT* __restrict__ keys, int64_t n, int shift,
                                                           int n_tiles, int* __restrict__ hist) {
    __shared__ int wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * RS_WARP_KEYS;
    const unsigned lt = lanemask_lt();
    // warp-aggregated: the leader of each group of equal digits adds the group's size
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t k = wbase + r * 32 + lane;
        const bool ok = k < n;
        const int d = ok ? (int)((keys[k] >> shift) & 255u) : 256 + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && (peers & lt) == 0) wcnt[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int c = 0;
#pragma unroll
        for (int q = 0; q < RS_WARPS; ++q) c += wcnt[q][d];
        hist[(int64_t)d * n_tiles + blockIdx.x] = c;
    }
}

template <class KT>
__global__ void __launch_bounds__(RS_WARPS * 32) k_rs_scatter(const KT* __restrict__ keys,
                                                              const uint32_t* __restrict__ vals, int64_t n, int shift,
                                                              int n_tiles, const int* __restrict__ offs,
                                                              KT* __restrict__ keys_out,
                                                              uint32_t* __restrict__ vals_out) {
    __shared__ int wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * RS_WARP_KEYS;
    KT kk[RS_ITEMS];
    uint32_t vv[RS_ITEMS];
    int dd[RS_ITEMS];
    const unsigned lt = lanemask_lt();
    // counts of the warp's sub-tile per digit (the leader of each group of equal digits adds)
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t k = wbase + r * 32 + lane;
        const bool ok = k < n;
        kk[r] = ok ? keys[k] : (KT)0;
        vv[r] = (ok && vals) ? vals[k] : 0u;
        dd[r] = ok ? (int)((kk[r] >> shift) & 255u) : 256 + lane;   // past the end: unique, never written
        const unsigned peers = __match_any_sync(0xffffffffu, dd[r]);
        if (ok && (peers & lt) == 0) wcnt[w][dd[r]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: global base of this tile plus the counts of the earlier warps
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        int run = offs[(int64_t)d * n_tiles + blockIdx.x];
#pragma unroll
        for (int q = 0; q < RS_WARPS; ++q) {
            const int c = wcnt[q][d];
            wcnt[q][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t k = wbase + r * 32 + lane;
        const bool ok = k < n;
        const unsigned peers = __match_any_sync(0xffffffffu, dd[r]);
        if (ok) {
            const int pos = wcnt[w][dd[r]] + __popc(peers & lt);
            keys_out[pos] = kk[r];
            if (vals_out) vals_out[pos] = vv[r];
        }
        __syncwarp();
        if (ok && (peers & lt) == 0) wcnt[w][dd[r]] += __popc(peers);
        __syncwarp();
    }
}

int64_t radix_sort_tiles(int64_t n) { return (n + RS_TILE - 1) / RS_TILE; }

size_t radix_sort_hist_ints(int64_t n) { return (size_t)256 * (size_t)radix_sort_tiles(n) + 1; }

// Sorts keys[0, n) (and vals with them, when vals is not NULL) by the low `bits` bits of the
// keys, ping-ponging with the alt arrays; on return *in_alt tells which holds the result.
// hist: radix_sort_hist_ints(n) ints; scan_tmp: scan_tmp_ints(radix_sort_hist_ints(n)) ints.
template <class KT>
int radix_sort(KT* keys, uint32_t* vals, KT* keys_alt, uint32_t* vals_alt, int64_t n, int bits, int* hist,
               int* scan_tmp, cudaStream_t st, bool* in_alt) {
    *in_alt = false;
    if (n <= 1 || bits <= 0) return WP_OK;
    const int64_t tiles = radix_sort_tiles(n);
    if (tiles > 2147483647LL / 256) return WP_ERR_SIZE;
    KT *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals ? vals_alt : nullptr;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<KT><<<(unsigned)tiles, RS_WARPS * 32, 0, st>>>(ka, n, shift, (int)tiles, hist);
        WP_LAUNCH_CHECK("k_rs_hist");
        int rc = exclusive_scan_i32(hist, hist, 256 * tiles, scan_tmp, st);
        if (rc) return rc;
        k_rs_scatter<KT><<<(unsigned)tiles, RS_WARPS * 32, 0, st>>>(ka, va, n, shift, (int)tiles, hist, kb, vb);
        WP_LAUNCH_CHECK("k_rs_scatter");
        KT* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
        *in_alt = !*in_alt;
    }
    return WP_OK;
}

template int radix_sort<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t, int, int*, int*, cudaStream_t,
                                  bool*);
template int radix_sort<uint64_t>(uint64_t*, uint32_t*, uint64_t*, uint32_t*, int64_t, int, int*, int*, cudaStream_t,
                                  bool*);

}  // namespace wp
