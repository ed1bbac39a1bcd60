// Hankel transform on the 5th-generation tensor cores (Section 4.3: the discrete transform
// is a matrix times a vector; all planes together make one matrix product).
//
//   C[m][n] = sum_k H[m][k] F[n][k],  m < K_out (radial output), n < 2 P_pad (re/im of each
//   plane), k < R_pad (radial input).
//
// Precision: TF32 inputs carry 11 significant bits, so each operand is split into
// hi = rna_tf32(x) and lo = rna_tf32(x - hi); the product is hi*hi' + hi*lo' + lo*hi'
// (the lo*lo' term is below 2^-22 relative), accumulated in FP32 in tensor memory.  The
// BF16 variant splits into two BF16 values (8 bits each: the three products then carry an
// operand error near 2^-17, measured 2e-6 relative on the transform) and runs kind::f16,
// twice the TF32 rate: a 128-byte swizzle row holds 64 BF16 elements instead of 32 TF32
// ones, and each MMA consumes 16 of them instead of 8 -- the same 32 bytes -- so the tile
// layout, descriptors and issue loop are shared and only the K depth per stage doubles.
// The BF16x6 variant splits each operand into three BF16 parts x = x0 + x1 + x2 (24
// significant bits, all of an FP32 value) and keeps the six products of order <= 2,
// x0 y0 + (x0 y1 + x1 y0) + (x0 y2 + x1 y1 + x2 y0), issued smallest first; the dropped
// terms are below 2^-24 relative, so it matches TF32x3's accuracy at the same tensor time
// (six products at twice the rate) with 6 instead of 8 operand bytes per element.
//
// Structure (one CTA = one 128 x 128 output tile, optionally one half of K):
//   warp 0 lane 0   TMA producer: per 128-byte K slice loads the split parts of A and B
//                   (A_hi, A_lo, B_hi, B_lo; three parts each for BF16x6; 128 rows x 128 B
//                   per tile, 128-byte swizzle) into a 3-stage ring (2 stages for BF16x6)
//   warp 1 lane 0   MMA issuer: 4 K-steps x 3 (or 6) products of tcgen05.mma (M = 128,
//                   N = 128, K = 8 TF32 or 16 BF16) per slice into one of two TMEM buffers,
//                   commits each stage back to the producer and each group of slices
//                   to the accumulation warps
//   warps 2-5       accumulation: tcgen05.ld of each finished partial (warp w reads TMEM
//                   lanes 32 (w % 4) ..) into FP32 registers; epilogue: column pairs
//                   (2p, 2p+1) stored as the complex radial sample of plane p (coalesced
//                   along the radial index)
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel records
// WP_ERR_TIMEOUT in `status`, stops issuing, drains what it issued, frees TMEM and returns.
// A drain that itself runs out of budget (a copy or MMA still in flight at exit) records
// WP_ERR_INFLIGHT instead, which callers must treat as a suspect context.
// `withhold_loads` (self-test only) keeps the producer idle so that the first wait expires.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "wp_internal.cuh"

namespace wp {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 32;           // BK fp32 = 128 bytes = one swizzle row
constexpr int BK16 = 64;                             // BF16 elements per 128-byte swizzle row
constexpr int TILE_BYTES = BM * BK * 4;              // 16 KB (BN == BM), either element type
constexpr int TMEM_COLS = 2 * BN;                   // two accumulator buffers

// Per-route configuration: MODE 0 = TF32x3, 1 = BF16x3, 2 = BF16x6.
template <int MODE>
struct Cfg {
    static constexpr bool BF16 = MODE != 0;
    static constexpr int NT = (MODE == 2) ? 3 : 2;                   // split parts per operand
    static constexpr int KS = BF16 ? BK16 : BK;                      // K elements per stage
    static constexpr int STAGES = (MODE == 2) ? 2 : 3;               // 2 x 96 KB or 3 x 64 KB
    static constexpr int STAGE_BYTES = 2 * NT * TILE_BYTES;          // A parts, then B parts
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    // K-slices per TMEM partial sum: 24 MMAs per partial in every mode (2 slices x 4 steps x 3
    // products, or 1 x 4 x 6)
    static constexpr int GROUP = (MODE == 2) ? 1 : 2;
};
static_assert(Cfg<2>::SMEM_BYTES <= 232448, "BF16x6 stages exceed shared memory");
constexpr long long WAIT_BUDGET = 4000000000LL;      // ~2 s of SM clock per wait (default)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase with `parity` completed, false after the budget
// (SM clock cycles), with WP_ERR_TIMEOUT recorded in `status`.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status, long long budget) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) {
            atomicMin(status, WP_ERR_TIMEOUT);   // the most severe code recorded wins
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row atoms of
// 1024 bytes stacked along M/N (stride 1024 B), version field 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);            // start address
    d |= (uint64_t)1 << 16;                             // leading byte offset (unused, 16 B)
    d |= (uint64_t)(1024 >> 4) << 32;                   // stride byte offset
    d |= (uint64_t)1 << 46;                             // fixed 0b001
    d |= (uint64_t)2 << 61;                             // swizzle: 128 B
    return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (format 1 for both: the two
// operands must share one type), both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

template <bool BF16>
__device__ __forceinline__ void mma_x(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (BF16) mma_bf16(tmem_d, a, b, idesc, acc);
    else mma_tf32(tmem_d, a, b, idesc, acc);
}

// The split products of one 32-byte K step: a[i], b[i] are the descriptors of part i.
// Two parts: hi*lo' + lo*hi' + hi*hi'; three parts: the six products of order <= 2, smallest
// first.  `acc0` = 0 starts a fresh accumulator with the first product.
template <int MODE>
__device__ __forceinline__ void mma_split(uint32_t d, const uint64_t (&a)[3], const uint64_t (&b)[3], uint64_t adv,
                                          uint32_t idesc, uint32_t acc0) {
    constexpr bool BF = Cfg<MODE>::BF16;
    if (MODE == 2) {
        mma_x<BF>(d, a[2] + adv, b[0] + adv, idesc, acc0);
        mma_x<BF>(d, a[1] + adv, b[1] + adv, idesc, 1u);
        mma_x<BF>(d, a[0] + adv, b[2] + adv, idesc, 1u);
        mma_x<BF>(d, a[1] + adv, b[0] + adv, idesc, 1u);
        mma_x<BF>(d, a[0] + adv, b[1] + adv, idesc, 1u);
        mma_x<BF>(d, a[0] + adv, b[0] + adv, idesc, 1u);
    } else {
        mma_x<BF>(d, a[0] + adv, b[1] + adv, idesc, acc0);
        mma_x<BF>(d, a[1] + adv, b[0] + adv, idesc, 1u);
        mma_x<BF>(d, a[0] + adv, b[0] + adv, idesc, 1u);
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_x32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Six warps: 0 = TMA producer, 1 = MMA issuer (and TMEM owner), 2..5 = accumulation and
// epilogue (warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. output rows of that quarter).
// The tensor core's FP32 accumulation does not round to nearest: its error grows with the
// number of MMA steps folded into one accumulator (about 2^-25 of the running sum per
// step, one-signed).  So the MMA issuer accumulates only GROUP K-slices (24 MMAs) into one of two
// TMEM buffers; the accumulation warps move each finished partial into FP32 registers
// (IEEE adds) while the next group runs into the other buffer.
template <int MODE>
__global__ void __launch_bounds__(192, 1) k_hankel_tf32x3(const __grid_constant__ CUtensorMap map_a0,
                                                          const __grid_constant__ CUtensorMap map_a1,
                                                          const __grid_constant__ CUtensorMap map_a2,
                                                          const __grid_constant__ CUtensorMap map_b0,
                                                          const __grid_constant__ CUtensorMap map_b1,
                                                          const __grid_constant__ CUtensorMap map_b2,
                                                          int M, int K, int k_split, int P,
                                                          float2* __restrict__ radial, int use_atomic,
                                                          int* __restrict__ status, long long budget,
                                                          int withhold_loads) {
    using C = Cfg<MODE>;
    constexpr int STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES, NT = C::NT, GROUP = C::GROUP;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * STAGE_BYTES);
    // bars: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
    const uint32_t bar_full0 = smem_u32(bars);
    const uint32_t bar_empty0 = smem_u32(bars + STAGES);
    const uint32_t bar_accf0 = smem_u32(bars + 2 * STAGES);
    const uint32_t bar_acce0 = smem_u32(bars + 2 * STAGES + 2);
    const uint32_t bar_done = smem_u32(bars + 2 * STAGES + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    constexpr int KS = C::KS;                          // K elements per stage
    const int kchunk = K / k_split;
    const int kbeg = blockIdx.z * kchunk;
    const int nkb = kchunk / KS;
    const int ngroups = (nkb + GROUP - 1) / GROUP;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar_full0 + 8 * s, 1);
            mbar_init(bar_empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_accf0 + 8 * b, 1);
            mbar_init(bar_acce0 + 8 * b, 4);     // one arrival per accumulation warp
        }
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0 && !withhold_loads) {
            // ---------------- TMA producer ----------------
            int issued = 0;
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES;
                if (kb >= STAGES) ok = mbar_wait(bar_empty0 + 8 * s, ((kb / STAGES) - 1) & 1, status, budget);
                if (!ok) break;
                const uint32_t st = base + s * STAGE_BYTES;
                const uint32_t fb = bar_full0 + 8 * s;
                mbar_expect_tx(fb, STAGE_BYTES);
                const int x = kbeg + kb * KS;   // a multiple of KS: 128-byte aligned inner coordinate
                tma_load_2d(st + 0 * TILE_BYTES, &map_a0, x, m0, fb);
                tma_load_2d(st + 1 * TILE_BYTES, &map_a1, x, m0, fb);
                if (NT == 3) tma_load_2d(st + 2 * TILE_BYTES, &map_a2, x, m0, fb);
                tma_load_2d(st + (NT + 0) * TILE_BYTES, &map_b0, x, n0, fb);
                tma_load_2d(st + (NT + 1) * TILE_BYTES, &map_b1, x, n0, fb);
                if (NT == 3) tma_load_2d(st + (NT + 2) * TILE_BYTES, &map_b2, x, n0, fb);
                ++issued;
            }
            if (!ok) {
                // every issued slice must land before the CTA may exit; if one still has not
                // after another budget, the CTA exits with a copy in flight into its shared
                // memory, which is recorded as its own status (the context is then suspect)
                for (int kb = max(0, issued - STAGES); kb < issued; ++kb)
                    if (!mbar_wait(bar_full0 + 8 * (kb % STAGES), (kb / STAGES) & 1, status, budget)) {
                        atomicMin(status, WP_ERR_INFLIGHT);
                        break;
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = C::BF16 ? idesc_bf16(BM, BN) : idesc_tf32(BM, BN);
            bool ok = true;
            for (int g = 0; g < ngroups && ok; ++g) {
                const int b = g & 1;
                if (g >= 2) ok = mbar_wait(bar_acce0 + 8 * b, ((g >> 1) - 1) & 1, status, budget);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + (uint32_t)(b * BN);
                const int kb_end = min(nkb, (g + 1) * GROUP);
                for (int kb = g * GROUP; kb < kb_end; ++kb) {
                    const int s = kb % STAGES;
                    if (!mbar_wait(bar_full0 + 8 * s, (kb / STAGES) & 1, status, budget)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st = base + s * STAGE_BYTES;
                    uint64_t da[3], db[3];
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        const int tt = t < NT ? t : NT - 1;   // unused third part for two-part splits
                        da[t] = smem_desc_sw128(st + tt * TILE_BYTES);
                        db[t] = smem_desc_sw128(st + (NT + tt) * TILE_BYTES);
                    }
                    const uint32_t first = (kb == g * GROUP) ? 1u : 0u;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        // 8 tf32 or 16 bf16 = 32 bytes along K per MMA
                        const uint64_t adv = (uint64_t)((j * 32) >> 4);
                        mma_split<MODE>(dacc, da, db, adv, idesc, (first && j == 0) ? 0u : 1u);
                    }
                    mma_commit(bar_empty0 + 8 * s);
                }
                if (ok) mma_commit(bar_accf0 + 8 * b);
            }
            mma_commit(bar_done);   // fires once every issued MMA has completed
        }
    } else {
        // ---------------- accumulation + epilogue (warps 2..5) ----------------
        const int q = warp & 3;                         // TMEM lane quarter
        float acc[BN];
#pragma unroll
        for (int i = 0; i < BN; ++i) acc[i] = 0.0f;
        bool ok = true;
        for (int g = 0; g < ngroups; ++g) {
            const int b = g & 1;
            // warp-uniform decision: every lane polls, the warp proceeds only if all saw it
            if (!__all_sync(0xffffffffu, mbar_wait(bar_accf0 + 8 * b, (g >> 1) & 1, status, budget))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN);
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld_x32_nowait(trow + c0, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[c0 + i] += __uint_as_float(r[i]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_acce0 + 8 * b);
        }
        if (ok && *status == 0) {
            const int m = m0 + q * 32 + lane;
#pragma unroll
            for (int j = 0; j < BN; j += 2) {
                const int p = (n0 + j) >> 1;
                if (p < P && m < M) {
                    float2* dst = radial + (int64_t)p * M + m;
                    if (use_atomic) atomicAdd(dst, make_float2(acc[j], acc[j + 1]));
                    else *dst = make_float2(acc[j], acc[j + 1]);
                }
            }
        }
    }
    __syncwarp();
    // no MMA may still write TMEM when it is freed (if the wait gives up, that is recorded as
    // the in-flight status: the tensor memory is then freed under a running MMA)
    if (warp == 1 && lane == 0 && !mbar_wait(bar_done, 0, status, budget)) atomicMin(status, WP_ERR_INFLIGHT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// ------------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2D row-major matrix [rows][cols] (cols contiguous) of FP32 (box 32 cols x 128 rows) or
// BF16 (box 64 cols x 128 rows): 128 bytes per box row, 128-byte swizzle.  Base must be
// 16-byte aligned and the row pitch a multiple of 16 bytes.
int make_map(CUtensorMap* map, const void* ptr, int rows, int cols, bool bf16 = false) {
    auto enc = get_encode();
    if (!enc) {
        set_last_error("cuTensorMapEncodeTiled", "driver entry point unavailable");
        return WP_ERR_CUDA;
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * (bf16 ? 2u : 4u)};
    cuuint32_t box[2] = {(cuuint32_t)(bf16 ? BK16 : BK), (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<void*>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_last_error("cuTensorMapEncodeTiled", "encoding failed");
        return WP_ERR_CUDA;
    }
    return WP_OK;
}

}  // namespace tc

namespace {
template <int MODE>
int gemm_split(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st,
               long long budget, int withhold_loads) {
    using namespace tc;
    using C = Cfg<MODE>;
    constexpr int KS = C::KS;
    const int M = g.k_out, N = 2 * p_pad(P), K = g.r_pad;
    if (M % BM || N % BN || K % KS) {
        set_last_error("kg_gemm_split", "shape not tile aligned");
        return WP_ERR_SIZE;
    }
    CUtensorMap ma[3], mb[3];
    int rc;
    if (C::BF16) {
        if ((rc = make_map(&ma[0], w.hb_hi, M, K, true))) return rc;
        if ((rc = make_map(&ma[1], w.hb_lo, M, K, true))) return rc;
        if ((rc = make_map(&ma[2], w.hb_lo2, M, K, true))) return rc;
        if ((rc = make_map(&mb[0], w.fb_hi, N, K, true))) return rc;
        if ((rc = make_map(&mb[1], w.fb_lo, N, K, true))) return rc;
        if ((rc = make_map(&mb[2], w.fb_lo2, N, K, true))) return rc;
    } else {
        if ((rc = make_map(&ma[0], w.h_hi, M, K))) return rc;
        if ((rc = make_map(&ma[1], w.h_lo, M, K))) return rc;
        ma[2] = ma[1];   // no third part
        if ((rc = make_map(&mb[0], w.f_hi, N, K))) return rc;
        if ((rc = make_map(&mb[1], w.f_lo, N, K))) return rc;
        mb[2] = mb[1];
    }
    int dev = 0, sms = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one CTA per SM: split K in two when the output tiles alone leave SMs idle
    const int tiles = (M / BM) * (N / BN);
    const int split = (tiles < sms && (K / 2) % KS == 0) ? 2 : 1;
    WP_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    if (split > 1) WP_CUDA(cudaMemsetAsync(radial, 0, (size_t)P * M * sizeof(float2), st));
    // per call (cheap; the attribute belongs to the current device's context)
    WP_CUDA(cudaFuncSetAttribute(k_hankel_tf32x3<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
    dim3 grid(N / BN, M / BM, split);
    k_hankel_tf32x3<MODE><<<grid, 192, C::SMEM_BYTES, st>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], M, K, split,
                                                            P, radial, split > 1, status, budget, withhold_loads);
    WP_LAUNCH_CHECK("k_hankel_tf32x3");
    return WP_OK;
}
}  // namespace

int kg_gemm_tf32x3_ex(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st,
                      long long budget, int withhold_loads) {
    return gemm_split<0>(g, w, P, radial, status, st, budget, withhold_loads);
}

int kg_gemm_bf16x3(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st) {
    return gemm_split<1>(g, w, P, radial, status, st, tc::WAIT_BUDGET, 0);
}

int kg_gemm_bf16x6(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st) {
    return gemm_split<2>(g, w, P, radial, status, st, tc::WAIT_BUDGET, 0);
}

int kg_gemm_tf32x3(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st) {
    return kg_gemm_tf32x3_ex(g, w, P, radial, status, st, tc::WAIT_BUDGET, 0);
}

}  // namespace wp
