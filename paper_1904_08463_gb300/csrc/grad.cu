// Gradients of the visibility prediction  V = degrid(K(t), image_to_grid(I; t))  with
// respect to the model image I and the radial anti-aliasing taper t (the differentiable
// form of the gridding / degridding pair of Alg. 1-2, with the kernels of Section 4.3).
//
// Convention: for a real loss L and complex V the incoming gradient is
// g = dL/dRe(V) + j dL/dIm(V); the gradient of a complex parameter z is returned in the
// same form, so that dL = Re(conj(g_z) dz).
//
//   k_grad_items     per-plane chunks of the binned visibilities (work items)
//   k_grad_radial    per visibility and tap: Q = conj(g) G(cell) (w >= 0) or g conj(G(cell))
//                    (w < 0, the kernel there is conjugated), scattered onto the radial line
//                    through the resample interpolation weights: d/dC_k gets b Q, d/dC_k+1
//                    gets a Q, and the spline second derivatives get the cubic weights;
//                    accumulated per plane in shared memory, flushed once per work item
//   k_spline_adjoint dC += D^T 6 A^-T dM (the spline system's adjoint, banded inverse),
//                    written as real/imaginary rows for the transposed product
//   k_gemm_nn        dF = dC H  (the Hankel transform's adjoint: the same matrix, transposed)
//   k_taper_kernels  dL/dt_i += sum_p Re(conj(dF_p,i) s_p,i),  s = exp(+2 pi j w_p (n_i - 1))
//   k_image_adjoint  after the inverse transform of grid(g): U = Re(centred IDFT) per pixel,
//                    dL/dI = U / (t wsum) inside the circle, and the pixel's
//                    dL/dt(r) = -U I / (t^2 wsum) spread onto the taper nodes through the
//                    linear-interpolation weights (shared-memory histogram)
#include <cuda_runtime.h>
#include <cufft.h>

#include "wp_internal.cuh"

namespace wp {

namespace {
constexpr int GCH = 256;           // visibilities per gradient work item
constexpr int GG_M = 128, GG_N = 128, GG_K = 32;
}  // namespace

// Work items: for plane p, ceil(n_p / GCH) chunks of its binned visibilities.
__global__ void k_grad_items(int P, int ntiles, const int* __restrict__ start, int* __restrict__ item_plane,
                             int* __restrict__ item_chunk, int* __restrict__ ctrl) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int n = 0;
    for (int p = 0; p < P; ++p) {
        const int cnt = start[(p + 1) * ntiles] - start[p * ntiles];
        const int ch = (cnt + GCH - 1) / GCH;
        for (int c = 0; c < ch; ++c) {
            item_plane[n] = p;
            item_chunk[n] = c;
            ++n;
        }
    }
    ctrl[0] = 0;   // item cursor
    ctrl[1] = n;   // item count
}

__global__ void __launch_bounds__(256) k_grad_radial(int N, int os, int s_max, int K, int ntiles,
                                                     const int32_t* __restrict__ support,
                                                     const int* __restrict__ start,
                                                     const int4* __restrict__ srec,
                                                     const float2* __restrict__ gvis,
                                                     const float2* __restrict__ grid,
                                                     const int* __restrict__ item_plane,
                                                     const int* __restrict__ item_chunk,
                                                     int* __restrict__ ctrl, float2* __restrict__ gC,
                                                     float2* __restrict__ gM, int cubic) {
    extern __shared__ float2 acc[];    // [2][K]: d/dC then d/dM of the current plane
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n_items = ctrl[1];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl[0], 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const int p = item_plane[it];
        const int S = min(max(support[p], 1), s_max);
        const int W = 2 * S + 1, W2 = W * W;
        const int lim = os * S, lim2 = lim * lim;
        const int ku = min(K, lim + 2);
        for (int k = threadIdx.x; k < 2 * ku; k += blockDim.x) acc[k] = make_float2(0.0f, 0.0f);
        __syncthreads();
        const int pb = start[p * ntiles], pe = start[(p + 1) * ntiles];
        const int r0 = pb + item_chunk[it] * GCH;
        const int r1 = min(pe, r0 + GCH);
        const float inv_w = 1.0f / (float)W;
        for (int r = r0 + wid; r < r1; r += 8) {
            const int4 r4 = srec[r];
            const int iu = r4.x & 0xffff, iv = (r4.x >> 16) & 0xffff;
            const int fu = r4.y & 0xff, fv = (r4.y >> 8) & 0xff;
            const bool neg = (r4.y >> 16) & 1;
            const float2 g = gvis[r4.w];
            const float2* g0 = grid + (int64_t)(iv - S) * N + (iu - S);
            for (int t = lane; t < W2; t += 32) {
                int jy = (int)(((float)t + 0.5f) * inv_w);
                jy -= (jy * W > t);
                jy += ((jy + 1) * W <= t);
                const int jx = t - jy * W;
                const int dx = os * (jx - S) - fu, dy = os * (jy - S) - fv;
                const int q = dx * dx + dy * dy;
                if (q > lim2) continue;                       // tap forced to zero: no gradient
                const float2 G = g0[(int64_t)jy * N + jx];
                float2 Q;
                if (!neg) Q = make_float2(g.x * G.x + g.y * G.y, g.x * G.y - g.y * G.x);   // conj(g) G
                else      Q = make_float2(g.x * G.x + g.y * G.y, g.y * G.x - g.x * G.y);   // g conj(G)
                const float x = sqrtf((float)q);
                const int k = min((int)x, K - 2);
                const float a = x - (float)k, b = 1.0f - a;
                atomicAdd(&acc[k].x, b * Q.x);
                atomicAdd(&acc[k].y, b * Q.y);
                atomicAdd(&acc[k + 1].x, a * Q.x);
                atomicAdd(&acc[k + 1].y, a * Q.y);
                if (cubic) {
                    const float cb = (b * b * b - b) * (1.0f / 6.0f);
                    const float ca = (a * a * a - a) * (1.0f / 6.0f);
                    atomicAdd(&acc[ku + k].x, cb * Q.x);
                    atomicAdd(&acc[ku + k].y, cb * Q.y);
                    atomicAdd(&acc[ku + k + 1].x, ca * Q.x);
                    atomicAdd(&acc[ku + k + 1].y, ca * Q.y);
                }
            }
        }
        __syncthreads();
        float2* dC = gC + (int64_t)p * K;
        float2* dM = gM + (int64_t)p * K;
        for (int k = threadIdx.x; k < ku; k += blockDim.x) {
            const float2 c = acc[k];
            if (c.x != 0.0f || c.y != 0.0f) atomicAdd(dC + k, c);
            if (cubic) {
                const float2 m = acc[ku + k];
                if (m.x != 0.0f || m.y != 0.0f) atomicAdd(dM + k, m);
            }
        }
        __syncthreads();
    }
}

// dC_total = dC + D^T (6 A^-T dM), written as rows 2p (re) and 2p + 1 (im) of gct [2 P_pad][K].
// band[d][k] = A^-1[k][k + d - 32].  D: row 0 = (C1 - C0), rows 1..K-2 = second differences,
// row K-1 = 0.
__global__ void __launch_bounds__(256) k_spline_adjoint(int K, int P, int cubic, const float* __restrict__ band,
                                                        const float2* __restrict__ gC,
                                                        const float2* __restrict__ gM,
                                                        float* __restrict__ gct) {
    extern __shared__ float2 sm[];     // gM[K], gR[K]
    float2* m = sm;
    float2* r = sm + K;
    const int p = blockIdx.x;
    float* ore = gct + (int64_t)(2 * p) * K;
    float* oim = ore + K;
    if (p >= P) {   // padded planes: zero rows
        for (int k = threadIdx.x; k < K; k += blockDim.x) { ore[k] = 0.0f; oim[k] = 0.0f; }
        return;
    }
    const float2* c = gC + (int64_t)p * K;
    if (!cubic) {
        for (int k = threadIdx.x; k < K; k += blockDim.x) { ore[k] = c[k].x; oim[k] = c[k].y; }
        return;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) m[k] = gM[(int64_t)p * K + k];
    __syncthreads();
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        float sr = 0.0f, si = 0.0f;
        for (int k = max(0, j - 32); k <= min(K - 1, j + 32); ++k) {
            const float w = band[(int64_t)(j - k + 32) * K + k];   // A^-1[k][j]
            sr = fmaf(w, m[k].x, sr);
            si = fmaf(w, m[k].y, si);
        }
        r[j] = make_float2(6.0f * sr, 6.0f * si);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float2 v = c[k];
        if (k == 0) { v.x -= r[0].x; v.y -= r[0].y; }
        if (k == 1) { v.x += r[0].x; v.y += r[0].y; }
        if (k - 1 >= 1 && k - 1 <= K - 2) { v.x += r[k - 1].x; v.y += r[k - 1].y; }
        if (k >= 1 && k <= K - 2) { v.x -= 2.0f * r[k].x; v.y -= 2.0f * r[k].y; }
        if (k + 1 >= 1 && k + 1 <= K - 2) { v.x += r[k + 1].x; v.y += r[k + 1].y; }
        ore[k] = v.x;
        oim[k] = v.y;
    }
}

// D[m][n] = sum_k A[m][k] B[k][n]; A = gct [M = 2 P_pad][K], B = H [K][Nc] (Nc = r_pad,
// columns guarded), FP32 SIMT, 128 x 128 x 32 tiles, 8 x 8 per thread.
__global__ void __launch_bounds__(256) k_gemm_nn(int M, int Nc, int K, const float* __restrict__ A,
                                                 const float* __restrict__ B, float* __restrict__ D) {
    __shared__ __align__(16) float As[GG_K][GG_M + 4];
    __shared__ __align__(16) float Bs[GG_K][GG_N + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * GG_M, n0 = blockIdx.x * GG_N;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += GG_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;
            const int row = e / 8, kq = (e % 8) * 4;
            const float4 a = *reinterpret_cast<const float4*>(A + (int64_t)(m0 + row) * K + k0 + kq);
            As[kq + 0][row] = a.x; As[kq + 1][row] = a.y; As[kq + 2][row] = a.z; As[kq + 3][row] = a.w;
            const int kr = e / 32, nc = (e % 32) * 4;
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n0 + nc < Nc) b = *reinterpret_cast<const float4*>(B + (int64_t)(k0 + kr) * Nc + n0 + nc);
            *reinterpret_cast<float4*>(&Bs[kr][nc]) = b;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GG_K; ++kk) {
            float a[8], b[8];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
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
        const int m = m0 + ty * 8 + i;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = n0 + tx * 8 + j;
            if (n < Nc) D[(int64_t)m * Nc + n] = acc[i][j];
        }
    }
}

// dL/dt_i += sum_p Re(conj(dF_p,i) s_p,i) with s the unit-modulus w-screen at node i.
__global__ void k_taper_kernels(int R, int r_pad, int P, const double* __restrict__ nm1,
                                const double* __restrict__ w_planes, const float* __restrict__ gF,
                                float* __restrict__ gt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    const double n1 = nm1[i];
    float sum = 0.0f;
    for (int p = 0; p < P; ++p) {
        const double cyc = w_planes[p] * n1;
        const double fr = cyc - rint(cyc);
        float s, c;
        sincospif((float)(2.0 * fr), &s, &c);
        const float fre = gF[(int64_t)(2 * p) * r_pad + i];
        const float fim = gF[(int64_t)(2 * p + 1) * r_pad + i];
        sum = fmaf(fre, c, fmaf(fim, s, sum));
    }
    gt[i] += sum;
}

// Image-domain adjoint after the inverse transform F of grid(g) (in place in `F`).
__global__ void __launch_bounds__(256) k_image_adjoint(int N, int R, const float* __restrict__ taper,
                                                       float inv_wsum, const float* __restrict__ image,
                                                       const float2* __restrict__ F,
                                                       float* __restrict__ grad_image,
                                                       float* __restrict__ gt) {
    extern __shared__ float hist[];   // [R]
    for (int i = threadIdx.x; i < R; i += blockDim.x) hist[i] = 0.0f;
    __syncthreads();
    const int h = N / 2;
    const int64_t npix = (int64_t)N * N;
    for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < npix;
         pix += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(pix / N), l = (int)(pix - (int64_t)m * N);
        const int dl_ = l - h, dm_ = m - h;
        const int d2 = dl_ * dl_ + dm_ * dm_;
        float gi = 0.0f;
        if (d2 <= h * h) {
            float U = F[(int64_t)((m + h) % N) * N + ((l + h) % N)].x;
            if ((l + m) & 1) U = -U;
            float x = 2.0f * (float)R * sqrtf((float)d2) / (float)N - 0.5f;
            x = fminf(fmaxf(x, 0.0f), (float)(R - 1));
            const int i0 = min((int)x, R - 2);
            const float a = x - (float)i0;
            const float t = (1.0f - a) * taper[i0] + a * taper[i0 + 1];
            gi = U * inv_wsum / t;
            const float gtp = -gi * image[pix] / t;   // d/dt of I / (t wsum), times U
            atomicAdd(&hist[i0], (1.0f - a) * gtp);
            atomicAdd(&hist[i0 + 1], a * gtp);
        }
        grad_image[pix] = gi;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x)
        if (hist[i] != 0.0f) atomicAdd(&gt[i], hist[i]);
}

// ------------------------------------------------------------------------------ launchers
size_t grad_extra_ints(int P, int64_t V) { return (size_t)(P + V / GCH + 2); }

int grad_radial_run(const Geom& g, const wp_wkernels* kern, const GridWork& w, int* item_plane, int* item_chunk,
                    const float2* gvis, const float2* grid, float2* gC, float2* gM, cudaStream_t st) {
    const int P = kern->P;
    WP_CUDA(cudaMemsetAsync(gC, 0, sizeof(float2) * (size_t)P * g.k_out, st));
    if (g.interp == WP_INTERP_CUBIC) WP_CUDA(cudaMemsetAsync(gM, 0, sizeof(float2) * (size_t)P * g.k_out, st));
    k_grad_items<<<1, 32, 0, st>>>(P, w.ntiles, w.count, item_plane, item_chunk, w.ctrl);
    WP_LAUNCH_CHECK("k_grad_items");
    int dev = 0, sms = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ku = g.os * g.s_max + 2 < g.k_out ? g.os * g.s_max + 2 : g.k_out;
    const size_t smem = (size_t)2 * ku * sizeof(float2);
    if (smem > 48 * 1024)
        WP_CUDA(cudaFuncSetAttribute(k_grad_radial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_grad_radial<<<sms * 4, 256, smem, st>>>(g.N, g.os, g.s_max, g.k_out, w.ntiles, kern->support, w.count, w.srec,
                                              gvis, grid, item_plane, item_chunk, w.ctrl, gC, gM,
                                              g.interp == WP_INTERP_CUBIC);
    WP_LAUNCH_CHECK("k_grad_radial");
    return WP_OK;
}

int hankel_adjoint_run(const Geom& g, const KgWork& w, int P, const double* w_planes, const float2* gC,
                       const float2* gM, float* grad_taper, cudaStream_t st) {
    const int Pp = p_pad(P);
    const int K = g.k_out;
    size_t smem = (size_t)2 * K * sizeof(float2);
    if (smem > 48 * 1024)
        WP_CUDA(cudaFuncSetAttribute(k_spline_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_spline_adjoint<<<Pp, 256, smem, st>>>(K, P, g.interp == WP_INTERP_CUBIC, w.band, gC, gM, w.gct);
    WP_LAUNCH_CHECK("k_spline_adjoint");
    dim3 grid((g.r_pad + GG_N - 1) / GG_N, (2 * Pp) / GG_M);
    k_gemm_nn<<<grid, 256, 0, st>>>(2 * Pp, g.r_pad, K, w.gct, w.h32, w.f32);
    WP_LAUNCH_CHECK("k_gemm_nn");
    k_taper_kernels<<<(g.R + 255) / 256, 256, 0, st>>>(g.R, g.r_pad, P, w.nm1, w_planes, w.f32, grad_taper);
    WP_LAUNCH_CHECK("k_taper_kernels");
    return WP_OK;
}

int launch_image_adjoint(const Geom& g, const float* taper, const float* image, const float2* F, double wsum,
                         float* grad_image, float* grad_taper, cudaStream_t st) {
    int dev = 0, sms = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = (size_t)g.R * sizeof(float);
    if (smem > 48 * 1024)
        WP_CUDA(cudaFuncSetAttribute(k_image_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_image_adjoint<<<sms * 4, 256, smem, st>>>(g.N, g.R, taper, (float)(1.0 / wsum), image, F, grad_image,
                                                grad_taper);
    WP_LAUNCH_CHECK("k_image_adjoint");
    return WP_OK;
}

}  // namespace wp
