// Kernel generation on the radial line (Section 4.3 of the paper, Alg. 2):
//   K1 j0 matrix   H[k][i] = du^2 2 pi r_i dr J0(2 pi rho_k r_i)   (FP64 evaluation, once)
//   K2 screen      f_p(r_i) = t(r_i) exp(+2 pi j w_p (sqrt(1 - r_i^2) - 1)) (FP64 phase)
//   K4 fp32 gemm   C = H F (FP32 SIMT matrix product, the plain comparator)
//   K5/K6          1 % truncation support and cubic-spline second derivatives
//   K7 resample    oversampled 2D kernel cache from the radial line
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "wp_internal.cuh"

namespace wp {

// =======================================================================================
// K1: transform matrix, built once per geometry (Section 4.3: it does not depend on the plane).
// With du * r_max = 1/2 the argument and weight reduce to integers times constants:
//   2 pi rho_k r_i = pi k (2i + 1) / (2 os R),   du^2 2 pi r_i dr = pi (2i + 1) / (4 R^2).
// The TF32 split keeps hi = rna_tf32(h), lo = rna_tf32(h - hi) so that
// hi*hi' + hi*lo' + lo*hi' reproduces the FP32 product to ~2^-22.
// =======================================================================================
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// x split as hi + lo with hi = bf16(x) and lo = bf16(x - hi), both round-to-nearest-even:
// together about 16 significant bits (the BF16x3 route's operands).  Each remainder is
// exact in FP32 (it holds the low bits of x).
__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

// Three-part split x = hi + lo + lo2 (the BF16x6 route's operands): lo2 = bf16 of what the
// pair leaves, so the three parts carry all 24 bits of the FP32 value.
__device__ __forceinline__ void split_bf16_3(float x, uint16_t& hi, uint16_t& lo, uint16_t& lo2) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1);
    const __nv_bfloat16 l2 = __float2bfloat16_rn(r1 - __bfloat162float(l));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
    lo2 = __bfloat16_as_ushort(l2);
}

// BF16 split of an FP32 array into three parts (the transform matrix of the BF16 routes:
// BF16x3 reads the first two, BF16x6 all three; hi and lo are the pair split_bf16 gives).
__global__ void k_split_bf16(int64_t n, const float* __restrict__ x, uint16_t* __restrict__ hi,
                             uint16_t* __restrict__ lo, uint16_t* __restrict__ lo2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint16_t h, l, l2;
    split_bf16_3(x[i], h, l, l2);
    hi[i] = h;
    lo[i] = l;
    lo2[i] = l2;
}

__global__ void k_j0_matrix(int k_out, int R, int r_pad, int os, float* __restrict__ h32,
                            float* __restrict__ h_hi, float* __restrict__ h_lo) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = (int64_t)k_out * r_pad;
    if (idx >= total) return;
    int k = (int)(idx / r_pad);
    int i = (int)(idx - (int64_t)k * r_pad);
    float v = 0.0f;
    if (i < R) {
        double two_i1 = (double)(2 * i + 1);
        double arg = M_PI * ((double)k * two_i1) / (2.0 * (double)os * (double)R);
        double wgt = M_PI * two_i1 / (4.0 * (double)R * (double)R);
        v = (float)(wgt * j0(arg));
    }
    h32[idx] = v;
    float hi = to_tf32(v);
    h_hi[idx] = hi;
    h_lo[idx] = to_tf32(v - hi);
}

// Host: band of the inverse of the spline system matrix (rows: [2 1], [1 4 1] ..., [.. 1]),
// stored diagonal-major: band[d][k] = A^-1[k][k + d - 32] (consecutive k contiguous).
// Entries of the inverse decay like (2 - sqrt 3)^|k - j| = 0.268^|k - j|, so a half-width
// of 32 keeps everything above 1e-18 of the diagonal.
static void spline_band_host(int K, std::vector<float>& band) {
    const int HW = 32;
    band.assign((size_t)K * (2 * HW + 1), 0.0f);
    std::vector<double> sub(K, 0.0), dia(K, 0.0), sup(K, 0.0), cp(K), x(K), d(K);
    dia[0] = 2.0; sup[0] = 1.0;
    for (int k = 1; k < K - 1; ++k) { sub[k] = 1.0; dia[k] = 4.0; sup[k] = 1.0; }
    dia[K - 1] = 1.0;
    // forward factor (independent of the right-hand side)
    cp[0] = sup[0] / dia[0];
    std::vector<double> den(K);
    den[0] = dia[0];
    for (int k = 1; k < K; ++k) {
        den[k] = dia[k] - sub[k] * cp[k - 1];
        cp[k] = sup[k] / den[k];
    }
    for (int j = 0; j < K; ++j) {
        // solve A x = e_j
        for (int k = 0; k < K; ++k) {
            double rhs = (k == j) ? 1.0 : 0.0;
            d[k] = (rhs - (k > 0 ? sub[k] * d[k - 1] : 0.0)) / den[k];
        }
        x[K - 1] = d[K - 1];
        for (int k = K - 2; k >= 0; --k) x[k] = d[k] - cp[k] * x[k + 1];
        for (int k = j - HW; k <= j + HW; ++k) {
            if (k < 0 || k >= K) continue;
            band[(size_t)(j - k + HW) * K + k] = (float)x[k];
        }
    }
}

// n - 1 at the radial nodes, in FP64, without cancellation: -r^2 / (1 + sqrt(1 - r^2)); also
// split into a float pair hi + lo (hi = the nearest float, lo = the nearest float to the rest).
__global__ void k_nm1(int R, int r_pad, double r_max, double* __restrict__ nm1, float2* __restrict__ nm1f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r_pad) return;
    double v = 0.0;
    if (i < R) {
        double r = ((double)i + 0.5) * (r_max / (double)R);
        double r2 = r * r;
        v = -r2 / (1.0 + sqrt(1.0 - r2));
    }
    nm1[i] = v;
    const float hi = (float)v;
    nm1f[i] = make_float2(hi, (float)(v - (double)hi));
}

int kg_prepare(const Geom& g, const KgWork& w, cudaStream_t st) {
    k_nm1<<<(g.r_pad + 255) / 256, 256, 0, st>>>(g.R, g.r_pad, g.r_max, w.nm1, w.nm1f);
    WP_LAUNCH_CHECK("k_nm1");
    // the tables of every route (transform matrix as FP32, TF32 and BF16 pairs; the workspace
    // n - 1 table of the projection route), so that any kernelgen route runs on this workspace
    {
        int rc = kg_ps_prepare(g, w, st);
        if (rc) return rc;
        int64_t total = (int64_t)g.k_out * g.r_pad;
        int threads = 256;
        int64_t blocks = (total + threads - 1) / threads;
        k_j0_matrix<<<(unsigned)blocks, threads, 0, st>>>(g.k_out, g.R, g.r_pad, g.os, w.h32, w.h_hi,
                                                           w.h_lo);
        WP_LAUNCH_CHECK("k_j0_matrix");
        k_split_bf16<<<(unsigned)blocks, threads, 0, st>>>(total, w.h32, w.hb_hi, w.hb_lo, w.hb_lo2);
        WP_LAUNCH_CHECK("k_split_bf16");
    }
    std::vector<float> band;
    spline_band_host(g.k_out, band);
    WP_CUDA(cudaMemcpyAsync(w.band, band.data(), band.size() * sizeof(float),
                            cudaMemcpyHostToDevice, st));
    // the host vector must outlive the copy: pageable copies are staged before return
    WP_CUDA(cudaStreamSynchronize(st));
    return WP_OK;
}

// =======================================================================================
// K2: image-domain convolution function on the radial line, written transposed
// (row 2p = real part, row 2p+1 = imaginary part, R contiguous) as the B operand of the
// K-major matrix product.  The phase in cycles, w (n - 1), must keep FP32 accuracy after
// reduction to [-1/2, 1/2] even for |w| ~ 1e5 (hundreds of cycles).  It is formed from the
// float pairs w = w_hi + w_lo and n - 1 = n_hi + n_lo (the latter precomputed once per
// geometry from FP64): p = w_hi n_hi rounded, its exact rounding error fma(w_hi, n_hi, -p),
// plus the cross terms (w_lo n_lo, ~2^-48 of the phase, is dropped); subtracting rint(p) from
// p is exact, and one final rounding gives the reduced phase -- as accurate as the FP64
// product rounded to float, on the FP32 units (FP64 throughput is low on this part).
// =======================================================================================
// One block per plane: the plane's w is split once, then every thread takes pairs of
// consecutive radial samples (one 8-byte FP32 / TF32 store or one 4-byte BF16-pair store per
// row and part), which keeps the per-plane latency chain short and the stores wide.
// MODE 0: FP32 rows (SIMT product); 1: TF32 hi/lo rows; 2: BF16 hi/lo rows; 3: BF16
// hi/lo/lo2 rows.
constexpr int SC_THREADS = 256;

__device__ __forceinline__ float2 screen_value(int i, int R, bool live, float2 w, const float2* __restrict__ nm1f,
                                               const float* __restrict__ taper) {
    float re = 0.0f, im = 0.0f;
    if (live && i < R) {
        const float2 n = nm1f[i];
        const float ph = w.x * n.x;
        float pl = fmaf(w.x, n.x, -ph);               // exact error of the high product
        pl = fmaf(w.x, n.y, fmaf(w.y, n.x, pl));      // cross terms
        const float fr = (ph - rintf(ph)) + pl;       // phase / (2 pi), reduced
        float sn, cs;
        sincospif(2.0f * fr, &sn, &cs);
        const float t = taper[i];
        re = t * cs;
        im = t * sn;
    }
    return make_float2(re, im);
}

__device__ __forceinline__ uint32_t pack_bf16(uint16_t a, uint16_t b) { return (uint32_t)a | ((uint32_t)b << 16); }

template <int MODE>
__global__ void __launch_bounds__(SC_THREADS) k_screen(int R, int r_pad, int P, const float2* __restrict__ nm1f,
                                                       const float* __restrict__ taper,
                                                       const double* __restrict__ w_planes,
                                                       float* __restrict__ f32, float* __restrict__ f_hi,
                                                       float* __restrict__ f_lo, uint16_t* __restrict__ fb_hi,
                                                       uint16_t* __restrict__ fb_lo, uint16_t* __restrict__ fb_lo2) {
    const int p = blockIdx.x;
    const bool live = p < P;
    const double wd = live ? w_planes[p] : 0.0;
    const float whi = (float)wd;
    const float2 w = make_float2(whi, (float)(wd - (double)whi));
    const int64_t row_re = (int64_t)(2 * p) * r_pad;
    const int64_t row_im = row_re + r_pad;
    for (int i = 2 * (int)threadIdx.x; i < r_pad; i += 2 * SC_THREADS) {   // r_pad is even
        const float2 v0 = screen_value(i, R, live, w, nm1f, taper);
        const float2 v1 = screen_value(i + 1, R, live, w, nm1f, taper);
        if (MODE == 1) {
            const float hr0 = to_tf32(v0.x), hr1 = to_tf32(v1.x), hi0 = to_tf32(v0.y), hi1 = to_tf32(v1.y);
            *reinterpret_cast<float2*>(f_hi + row_re + i) = make_float2(hr0, hr1);
            *reinterpret_cast<float2*>(f_hi + row_im + i) = make_float2(hi0, hi1);
            *reinterpret_cast<float2*>(f_lo + row_re + i) = make_float2(to_tf32(v0.x - hr0), to_tf32(v1.x - hr1));
            *reinterpret_cast<float2*>(f_lo + row_im + i) = make_float2(to_tf32(v0.y - hi0), to_tf32(v1.y - hi1));
        } else if (MODE == 2) {
            uint16_t a0, b0, a1, b1, c0, d0, c1, d1;
            split_bf16(v0.x, a0, b0);
            split_bf16(v1.x, a1, b1);
            split_bf16(v0.y, c0, d0);
            split_bf16(v1.y, c1, d1);
            *reinterpret_cast<uint32_t*>(fb_hi + row_re + i) = pack_bf16(a0, a1);
            *reinterpret_cast<uint32_t*>(fb_lo + row_re + i) = pack_bf16(b0, b1);
            *reinterpret_cast<uint32_t*>(fb_hi + row_im + i) = pack_bf16(c0, c1);
            *reinterpret_cast<uint32_t*>(fb_lo + row_im + i) = pack_bf16(d0, d1);
        } else if (MODE == 3) {
            uint16_t a0, b0, e0, a1, b1, e1, c0, d0, g0, c1, d1, g1;
            split_bf16_3(v0.x, a0, b0, e0);
            split_bf16_3(v1.x, a1, b1, e1);
            split_bf16_3(v0.y, c0, d0, g0);
            split_bf16_3(v1.y, c1, d1, g1);
            *reinterpret_cast<uint32_t*>(fb_hi + row_re + i) = pack_bf16(a0, a1);
            *reinterpret_cast<uint32_t*>(fb_lo + row_re + i) = pack_bf16(b0, b1);
            *reinterpret_cast<uint32_t*>(fb_lo2 + row_re + i) = pack_bf16(e0, e1);
            *reinterpret_cast<uint32_t*>(fb_hi + row_im + i) = pack_bf16(c0, c1);
            *reinterpret_cast<uint32_t*>(fb_lo + row_im + i) = pack_bf16(d0, d1);
            *reinterpret_cast<uint32_t*>(fb_lo2 + row_im + i) = pack_bf16(g0, g1);
        } else {
            *reinterpret_cast<float2*>(f32 + row_re + i) = make_float2(v0.x, v1.x);
            *reinterpret_cast<float2*>(f32 + row_im + i) = make_float2(v0.y, v1.y);
        }
    }
}

int kg_screen(const Geom& g, const KgWork& w, const float* taper, const double* w_planes, int P,
              cudaStream_t st) {
    const int Pp = p_pad(P);
    if (g.kernelgen == WP_KG_TF32X3)
        k_screen<1><<<Pp, SC_THREADS, 0, st>>>(g.R, g.r_pad, P, w.nm1f, taper, w_planes, w.f32, w.f_hi, w.f_lo,
                                               w.fb_hi, w.fb_lo, w.fb_lo2);
    else if (g.kernelgen == WP_KG_BF16X3)
        k_screen<2><<<Pp, SC_THREADS, 0, st>>>(g.R, g.r_pad, P, w.nm1f, taper, w_planes, w.f32, w.f_hi, w.f_lo,
                                               w.fb_hi, w.fb_lo, w.fb_lo2);
    else if (g.kernelgen == WP_KG_BF16X6)
        k_screen<3><<<Pp, SC_THREADS, 0, st>>>(g.R, g.r_pad, P, w.nm1f, taper, w_planes, w.f32, w.f_hi, w.f_lo,
                                               w.fb_hi, w.fb_lo, w.fb_lo2);
    else
        k_screen<0><<<Pp, SC_THREADS, 0, st>>>(g.R, g.r_pad, P, w.nm1f, taper, w_planes, w.f32, w.f_hi, w.f_lo,
                                               w.fb_hi, w.fb_lo, w.fb_lo2);
    WP_LAUNCH_CHECK("k_screen");
    return WP_OK;
}

// =======================================================================================
// K4: plain FP32 SIMT matrix product  D[m][n] = sum_k A[m][k] B[n][k]
//   A = H [M = k_out][K = r_pad], B = F^T [N = 2 P_pad][K], both K-contiguous.
// 128 x 128 block tile, 32-deep K slices through shared memory, 8 x 8 register tile per
// thread.  Output column n = 2p + c is component c of radial[p][m].  With split-K = 2
// the two halves are combined with atomicAdd into a zeroed output (two addends: the
// result does not depend on their order).
// =======================================================================================
namespace {
constexpr int GB_M = 128, GB_N = 128, GB_K = 32, GB_PAD = 4;
}

__global__ void __launch_bounds__(256) k_gemm_fp32(int M, int N, int K, int k_split,
                                                   const float* __restrict__ A,
                                                   const float* __restrict__ B, int P,
                                                   float2* __restrict__ radial, int use_atomic) {
    __shared__ __align__(16) float As[GB_K][GB_M + GB_PAD];
    __shared__ __align__(16) float Bs[GB_K][GB_N + GB_PAD];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    const int kchunk = K / k_split;
    const int kbeg = blockIdx.z * kchunk, kend = kbeg + kchunk;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
        // 128 rows x 32 k = 1024 float4 per operand, 4 per thread
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + q * 256;
            int row = e / 8, kq = (e % 8) * 4;
            float4 a = *reinterpret_cast<const float4*>(A + (int64_t)(m0 + row) * K + k0 + kq);
            float4 b = *reinterpret_cast<const float4*>(B + (int64_t)(n0 + row) * K + k0 + kq);
            As[kq + 0][row] = a.x; As[kq + 1][row] = a.y; As[kq + 2][row] = a.z; As[kq + 3][row] = a.w;
            Bs[kq + 0][row] = b.x; Bs[kq + 1][row] = b.y; Bs[kq + 2][row] = b.z; Bs[kq + 3][row] = b.w;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GB_K; ++kk) {
            float a[8], b[8];
            float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
            float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
            float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
            float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int m = m0 + ty * 8 + i;
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            int n = n0 + tx * 8 + j;
            int p = n >> 1;
            if (p < P) {
                float2* dst = radial + (int64_t)p * M + m;
                if (use_atomic) {
                    atomicAdd(&dst->x, acc[i][j]);
                    atomicAdd(&dst->y, acc[i][j + 1]);
                } else {
                    *dst = make_float2(acc[i][j], acc[i][j + 1]);
                }
            }
        }
    }
}

int kg_gemm_fp32(const Geom& g, const KgWork& w, int P, float2* radial, cudaStream_t st) {
    int M = g.k_out, N = 2 * p_pad(P), K = g.r_pad;
    int dev = 0, sms = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int tiles = (M / GB_M) * (N / GB_N);
    int split = (tiles < sms && (K / 2) % GB_K == 0) ? 2 : 1;
    if (split > 1) WP_CUDA(cudaMemsetAsync(radial, 0, (size_t)P * M * sizeof(float2), st));
    dim3 grid(N / GB_N, M / GB_M, split);
    k_gemm_fp32<<<grid, 256, 0, st>>>(M, N, K, split, w.h32, w.f32, P, radial, split > 1);
    WP_LAUNCH_CHECK("k_gemm_fp32");
    return WP_OK;
}

// =======================================================================================
// K5 + K6: per plane (one block): 1 % truncation support and spline second derivatives.
// Support: last k with |C_k| >= tau * max |C|, S = ceil(k / os) clamped to [S_min, S_max].
// Spline: m = A^-1 rhs with rhs_0 = 6 (y1 - y0), rhs_k = 6 (y_{k+1} - 2 y_k + y_{k-1}),
// rhs_{K-1} = 0 (zero slope at rho = 0, natural end), using the precomputed band of A^-1.
// The inverse of this diagonally dominant tridiagonal matrix decays like (2 - sqrt 3)^|k-j| =
// 0.268^|k-j| away from the diagonal, so the product keeps |k - j| <= 16 (the dropped tail is
// below 2e-10 of the largest coefficient, 300x under FP32 resolution of the sum); rows k with
// 16 <= k < K - 16 equal the interior (Toeplitz) row up to boundary reflections ~0.268^(2k),
// so only the 16 first and 16 last rows use their own coefficients.
// =======================================================================================
constexpr int TS_THREADS = 384;   // threads per plane of the truncation / spline kernel (3 rows each at K 1152)
constexpr int SPL_HW = 16;        // band half-width used by the product (the stored band holds 32)

__global__ void __launch_bounds__(TS_THREADS) k_trunc_spline(int K, int os, int s_min, int s_max, float tau,
                                                      int do_trunc, int do_spline,
                                                      const float2* __restrict__ radial,
                                                      const float* __restrict__ band,
                                                      float2* __restrict__ spline_m,
                                                      int32_t* __restrict__ support) {
    extern __shared__ float2 sm[];   // y[K], rhs[K + 64] (rhs padded by 32 zeros on each side)
    float2* y = sm;
    float2* rhs = sm + K + 32;
    __shared__ float red_f[TS_THREADS / 32];
    __shared__ int red_i[TS_THREADS / 32];
    constexpr int NB = 2 * SPL_HW + 1;              // band width used
    __shared__ float toe[NB];                       // the interior (Toeplitz) row, offsets -16..16
    __shared__ float edge[NB * 2 * SPL_HW];         // the 16 first and 16 last rows: edge[e * 32 + kk]
    const int p = blockIdx.x;
    if (do_spline) {
        // stored band row d holds A^-1[k][k + d - 32]; offsets -16..16 are d = 16..48
        if (threadIdx.x < NB) toe[threadIdx.x] = band[(int64_t)(threadIdx.x + 32 - SPL_HW) * K + K / 2];
        // staged by the whole block (coalesced along k); K >= 128
        for (int i = threadIdx.x; i < NB * 2 * SPL_HW; i += blockDim.x) {
            const int e = i / (2 * SPL_HW), kk = i - e * (2 * SPL_HW);
            edge[i] = band[(int64_t)(e + 32 - SPL_HW) * K + (kk < SPL_HW ? kk : K - 2 * SPL_HW + kk)];
        }
    }
    const float2* src = radial + (int64_t)p * K;
    float local_max = 0.0f;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float2 v = src[k];
        y[k] = v;
        local_max = fmaxf(local_max, sqrtf(v.x * v.x + v.y * v.y));
    }
    for (int k = threadIdx.x; k < 32; k += blockDim.x) {
        rhs[k - 32] = make_float2(0.0f, 0.0f);
        rhs[K + k] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (do_trunc) {
        for (int o = 16; o; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        if (lane == 0) red_f[wid] = local_max;
        __syncthreads();
        float mx = 0.0f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) mx = fmaxf(mx, red_f[q]);
        float thr = tau * mx;
        int last = 0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            float2 v = y[k];
            if (sqrtf(v.x * v.x + v.y * v.y) >= thr) last = max(last, k);
        }
        for (int o = 16; o; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
        if (lane == 0) red_i[wid] = last;
        __syncthreads();
        if (threadIdx.x == 0) {
            int kl = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) kl = max(kl, red_i[q]);
            int s = (kl + os - 1) / os;
            s = min(max(s, s_min), s_max);
            support[p] = s;
        }
    }
    if (do_spline) {
        for (int j = threadIdx.x; j < K; j += blockDim.x) {
            float2 r;
            if (j == 0) {
                r = make_float2(6.0f * (y[1].x - y[0].x), 6.0f * (y[1].y - y[0].y));
            } else if (j == K - 1) {
                r = make_float2(0.0f, 0.0f);
            } else {
                r = make_float2(6.0f * ((y[j + 1].x - y[j].x) - (y[j].x - y[j - 1].x)),
                                6.0f * ((y[j + 1].y - y[j].y) - (y[j].y - y[j - 1].y)));
            }
            rhs[j] = r;
        }
        __syncthreads();
        float2* dst = spline_m + (int64_t)p * K;
        float tr[NB];                               // the Toeplitz row in registers
#pragma unroll
        for (int e = 0; e < NB; ++e) tr[e] = toe[e];
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            float mr = 0.0f, mi = 0.0f;
            if (k >= SPL_HW && k < K - SPL_HW) {
#pragma unroll
                for (int e = 0; e < NB; ++e) {
                    const float2 r = rhs[k + e - SPL_HW];
                    mr = fmaf(tr[e], r.x, mr);
                    mi = fmaf(tr[e], r.y, mi);
                }
            } else {
                const int kk = k < SPL_HW ? k : k - (K - 2 * SPL_HW);
#pragma unroll
                for (int e = 0; e < NB; ++e) {
                    const float c = edge[e * 2 * SPL_HW + kk];   // zero where k + e - 16 is outside
                    const float2 r = rhs[k + e - SPL_HW];
                    mr = fmaf(c, r.x, mr);
                    mi = fmaf(c, r.y, mi);
                }
            }
            dst[k] = make_float2(mr, mi);
        }
    }
}

int kg_trunc_spline(const Geom& g, const KgWork& w, int P, const float2* radial, float2* spline_m,
                    int32_t* support, cudaStream_t st) {
    int do_trunc = (g.tau > 0.0) ? 1 : 0;
    int do_spline = (g.interp == WP_INTERP_CUBIC) ? 1 : 0;
    if (!do_trunc && !do_spline) return WP_OK;
    size_t smem = (size_t)(2 * g.k_out + 64) * sizeof(float2);
    // static staging (~17 KB) + dynamic can pass the 48 KB default from K ~ 1900 on
    WP_CUDA(cudaFuncSetAttribute(k_trunc_spline, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_trunc_spline<<<P, TS_THREADS, smem, st>>>(g.k_out, g.os, g.s_min, g.s_max, (float)g.tau, do_trunc,
                                         do_spline, radial, w.band, spline_m, support);
    WP_LAUNCH_CHECK("k_trunc_spline");
    return WP_OK;
}

// =======================================================================================
// K7: resample the radial line into the oversampled cache.
//
// Every tap of every sub-kernel samples one radially symmetric 2D function on the fine
// grid (spacing du/os): tap (jx, jy) of sub-kernel (fu, fv) sits at fine offset
// (dx, dy) = (os (jx - S) - fu, os (jy - S) - fv) and its value depends only on
// q = dx^2 + dy^2.  Negating dx maps sub-kernel fu onto fu' = (os - fu) mod os:
//   fu = 0    jx -> 2S - jx        (onto itself)
//   fu > 0    jx -> 2S + 1 - jx    (onto fu'; fu' = fu when 2 fu = os)
// and column jx = 0 of a sub-kernel with fu > 0 lies beyond the support radius
// (|dx| > os S): it is zero, and it is the image of column 0 of fu.  Likewise for y.
//
// One block per (plane, representative fu, fv <= os/2) evaluates each axis only over the
// part its mirror does not cover -- [0, S] when the sub-kernel is its own mirror
// (fu = 0 or 2 fu = os), [0, 2S] otherwise -- and stores every evaluated tap to four cache
// entries (neither, x, y, both mirrored); entries that coincide (centre lines, the zero
// line of 2 fu = os) receive the same bits twice, since the value is a function of q.
// For os = 8 that is (8S + 5)^2 evaluations for 64 (2S + 1)^2 cache entries.  Blocks are
// issued from the last plane backwards (supports grow with |w|: the largest blocks start
// first); consecutive threads take consecutive taps of the flattened evaluation domain, so
// each of the four stores of a warp covers contiguous runs of the cache.
//
// Tap values: the plane's line (value + spline second derivative, 16 B per sample) sits
// in shared memory with an XOR swizzle of the slot within each group of 8 (neighbouring
// taps are up to os samples apart on the line; the swizzle spreads them over the banks).
// The radius test q <= (os S)^2 is an exact integer test; x = sqrt(q) only picks the
// spline interval and its weights, which are continuous across interval ends.
// =======================================================================================
// skew() and resample_tap() live in wp_internal.cuh (the on-the-fly gridder uses them too).

// Bulk (TMA) store from shared memory: a byte range, 16-byte aligned on both sides and a
// multiple of 16 bytes long, written by the copy engine in whole cache lines.
__device__ __forceinline__ void bulk_store(float2* gdst, uint32_t saddr, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 ::"l"(gdst), "r"(saddr), "r"(bytes) : "memory");
}

__device__ __forceinline__ int parity8(const float2* g) { return (int)(((uintptr_t)g >> 3) & 1); }

constexpr int RS_THREADS = 512;   // 16 warps, two blocks per SM (384 and 576+ measured slower)

// Staged output: every chunk of whole evaluated rows [r0, r1) lands in at most four contiguous
// cache ranges -- rows [r0, r1) of the sub-kernel itself (F) and of its x-mirror (X), the
// mirrored rows of the y-mirror (Y) and of the xy-mirror (XY); when the sub-kernel is its own
// x-mirror, X and XY fold into F and Y.  Each range is assembled in shared memory, placed so
// that shared and global addresses agree modulo 16 bytes, and written by the copy engine
// (cp.async.bulk) in whole cache lines; an odd head / tail element goes through a plain store.
// Plain warp stores of these ranges would start 8 bytes off the 16-byte grid for every other
// sub-kernel and row, and run in reverse for the mirrors, which costs about a third of the
// write bandwidth.  Two buffer sets alternate with one barrier per chunk: before it, the
// threads that issued the copies of chunk c - 1 wait until those have read their set, which
// chunk c + 1 overwrites.
template <bool CUBIC>
__global__ void __launch_bounds__(RS_THREADS) k_resample(int K, int os, int s_max, int nrep, int n_items,
                                                         int n_line, int slot, int nsets,
                                                         const float2* __restrict__ radial,
                                                         const float2* __restrict__ spline_m,
                                                         const int32_t* __restrict__ support,
                                                         const int64_t* __restrict__ offsets,
                                                         float2* __restrict__ cache) {
    extern __shared__ float4 line[];   // skew(n_used) entries {y.re, y.im, m.re, m.im}, then
                                       // nsets (2, or 1 when two would cost a block per SM)
                                       // buffer sets x 4 regions x slot float2
    float2* const stage = reinterpret_cast<float2*>(line + n_line);
    const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(stage);
    const int item = n_items - 1 - (int)blockIdx.x;
    const int p = item / nrep;
    const int rep = item - p * nrep;
    const int h = os / 2;
    const int fv = rep / (h + 1), fu = rep - fv * (h + 1);   // 0 <= fu, fv <= os / 2
    // supports outside [1, S_max] are clamped, and to what the plane's block can hold
    const int S = fit_support(min(max(support[p], 1), s_max), os, offsets, p);
    if (S < 1) return;   // block-uniform, before any barrier
    const int W = 2 * S + 1;
    const int W2 = W * W;
    const int lim = os * S;
    const int n_used = min(K, lim + 2);
    const float2* yl = radial + (int64_t)p * K;
    const float2* ml = spline_m + (int64_t)p * K;
    for (int k = threadIdx.x; k < n_used; k += blockDim.x) {
        float2 a = yl[k];
        float2 b = CUBIC ? ml[k] : make_float2(0.0f, 0.0f);
        line[skew(k)] = make_float4(a.x, a.y, b.x, b.y);
    }
    // per axis: mirror sub-kernel, evaluated extent, mirror centre
    const int fu2 = fu ? os - fu : 0, fv2 = fv ? os - fv : 0;
    const bool xself = (fu2 == fu);
    const int nx = xself ? S + 1 : W, ny = (fv2 == fv) ? S + 1 : W;
    const int cx = fu ? W : W - 1, cy = fv ? W : W - 1;   // j -> c - j (j = 0 with f > 0: -> 0)
    float2* const base = cache + offsets[p];
    const int64_t blk = offsets[p + 1] - offsets[p];   // the plane's block (checked build)
    float2* const d00 = base + (int64_t)(fv * os + fu) * W2;
    float2* const d10 = base + (int64_t)(fv * os + fu2) * W2;    // x-mirrored
    float2* const d01 = base + (int64_t)(fv2 * os + fu) * W2;    // y-mirrored
    float2* const d11 = base + (int64_t)(fv2 * os + fu2) * W2;   // both
    const float2 zero = make_float2(0.0f, 0.0f);
    if (fv2 != fv)   // row 0 of the y-mirrored sub-kernels has no pre-image: zero
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            if (in_bounds((d01 - base) + i, blk, BS_CACHE_WRITE)) __stcs(d01 + i, zero);
            if (!xself && in_bounds((d11 - base) + i, blk, BS_CACHE_WRITE)) __stcs(d11 + i, zero);
        }
    const int lim2 = lim * lim;
    const int dy0 = -os * S - fv;   // os (jy - S) - fv at jy = 0
    const int dx0 = -os * S - fu;   // os (jx - S) - fu at jx = 0
    const int rpc = max(1, (slot - 2) / W);   // rows per chunk
    const int step_r = (int)blockDim.x / nx, step_c = (int)blockDim.x - step_r * nx;
    const int jy_t = (int)threadIdx.x / nx, jx_t = (int)threadIdx.x - jy_t * nx;
    __syncthreads();   // line staged
    int so = 0;        // offset of the current buffer set
    for (int r0 = 0, chunk = 0; r0 < ny; r0 += rpc, ++chunk) {
        const int r1 = min(ny, r0 + rpc);
        const int ya = (fv && r0 == 0) ? 1 : r0;   // rows with a y-mirror: [ya, r1)
        const int ylo = cy - (r1 - 1);              // lowest mirrored row
        float2* const gF = d00 + r0 * W;
        float2* const gX = d10 + r0 * W;
        float2* const gY = d01 + ylo * W;
        float2* const gXY = d11 + ylo * W;
        const int oF = so + parity8(gF);
        const int oX = xself ? oF : so + slot + parity8(gX);
        const int oY = so + 2 * slot + parity8(gY);
        const int oXY = xself ? oY : so + 3 * slot + parity8(gXY);
        if (nsets == 1 && chunk >= 1) {   // one set: chunk - 1's copies must have read it
            if (threadIdx.x < 4) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            __syncthreads();
        }
        int jy = r0 + jy_t, jx = jx_t;
        const int n_eval = (r1 - r0) * nx;
        for (int t = threadIdx.x; t < n_eval; t += blockDim.x) {
            const float2 v = resample_tap<CUBIC>(line, dx0 + os * jx, dy0 + os * jy, lim2);
            const int mj = (jx == 0 && fu) ? 0 : cx - jx;
            const int lf = (jy - r0) * W;
            // mirrored row cy - jy relative to ylo; the row jy = 0 without a mirror (fv > 0)
            // lands past the Y range's end and is never copied out
            const int lm = (r1 - 1 - jy) * W;
            stage[oF + lf + jx] = v;
            stage[oX + lf + mj] = v;
            stage[oY + lm + jx] = v;
            stage[oXY + lm + mj] = v;
            jx += step_c;
            jy += step_r;
            if (jx >= nx) { jx -= nx; ++jy; }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // threads 0..3 own one region's copies each; chunk - 1's must have read the other set
        if (threadIdx.x < 4 && chunk >= 1) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncthreads();
        if (threadIdx.x < 4) {
            const int k = threadIdx.x;
            const int nF = (r1 - r0) * W, nY = (r1 - ya) * W;
            float2* const g = k == 0 ? gF : k == 1 ? gX : k == 2 ? gY : gXY;
            const int o = k == 0 ? oF : k == 1 ? oX : k == 2 ? oY : oXY;
            const int n = k == 0 ? nF : k == 1 ? (xself ? 0 : nF) : k == 2 ? nY : (xself ? 0 : nY);
            if (n > 0 && in_bounds(g - base, blk, BS_CACHE_WRITE) && in_bounds((g - base) + n - 1, blk, BS_CACHE_WRITE)) {
                const int sh = parity8(g);          // odd head element
                const int nb = (n - sh) & ~1;       // aligned body
                if (nb > 0) bulk_store(g + sh, stage_s + 8u * (uint32_t)(o + sh), (uint32_t)nb * 8u);
                if (sh) __stcs(g, stage[o]);
                if ((n - sh) & 1) __stcs(g + (n - 1), stage[o + n - 1]);
            }
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        if (nsets == 2) so = so ? 0 : 4 * slot;
    }
    // bulk copies must finish reading shared memory before the block exits
    if (threadIdx.x < 4) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

int kg_resample(const Geom& g, int P, const float2* radial, const float2* spline_m,
                const int32_t* support, const int64_t* offsets, float2* cache, cudaStream_t st) {
    int n_max = g.os * g.s_max + 2;
    if (n_max > g.k_out) n_max = g.k_out;
    const int n_line = (int)round_up(n_max, 8);
    const size_t line_bytes = (size_t)n_line * sizeof(float4);
    // staging capacity per region (elements, even): up to 1536 -- three taps per thread per
    // chunk -- while two blocks still fit on an SM; never below one row of the largest
    // support
    int dev = 0, smem_sm = 0, smem_block = 0, reserved = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    WP_CUDA(cudaDeviceGetAttribute(&smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    WP_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    // (two buffer sets; when those would leave room for one block per SM but a single set
    // would not, one set and a second barrier per chunk -- large supports at high os)
    const int w_max = 2 * g.s_max + 1;
    const long two_per_sm = (long)smem_sm / 2 - reserved - (long)line_bytes;
    int nsets = 2;
    int cap = (int)(two_per_sm / (8 * (long)sizeof(float2))) - 2;
    if (cap < w_max + 1) {
        const int cap1 = (int)(two_per_sm / (4 * (long)sizeof(float2))) - 2;
        if (cap1 >= w_max + 1) {
            nsets = 1;
            cap = cap1;
        }
    }
    const int cap_max = (nsets == 2) ? 1536 : 3072;   // three (six) taps per thread per chunk
    cap = cap > cap_max ? cap_max : cap;
    cap &= ~1;
    if (cap < w_max + 1) cap = w_max + 1;   // even, >= one row
    const int slot = cap + 2;
    const size_t smem = line_bytes + (size_t)4 * nsets * slot * sizeof(float2);
    if (smem > (size_t)smem_block) {
        set_last_error("wp_resample", "staging for this support and oversampling exceeds shared memory");
        return WP_ERR_UNSUPPORTED;
    }
    const int h = g.os / 2;
    const int nrep = (h + 1) * (h + 1);
    const int n_items = P * nrep;
    dim3 grid((unsigned)n_items);
    if (g.interp == WP_INTERP_CUBIC) {
        WP_CUDA(cudaFuncSetAttribute(k_resample<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_resample<true><<<grid, RS_THREADS, smem, st>>>(g.k_out, g.os, g.s_max, nrep, n_items, n_line, slot, nsets,
                                                         radial, spline_m, support, offsets, cache);
    } else {
        WP_CUDA(cudaFuncSetAttribute(k_resample<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_resample<false><<<grid, RS_THREADS, smem, st>>>(g.k_out, g.os, g.s_max, nrep, n_items, n_line, slot, nsets,
                                                          radial, spline_m, support, offsets, cache);
    }
    WP_LAUNCH_CHECK("k_resample");
    return WP_OK;
}

}  // namespace wp
