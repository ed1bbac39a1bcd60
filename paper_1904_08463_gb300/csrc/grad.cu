// Gradients of the visibility prediction  V = degrid(K(t), image_to_grid(I; t))  with
// respect to the model image I and the radial anti-aliasing taper t (the differentiable
// form of the gridding / degridding pair of Alg. 1-2, with the kernels of Section 4.3).
//
// Convention: for a real loss L and complex V the incoming gradient is
// g = dL/dRe(V) + j dL/dIm(V); the gradient of a complex parameter z is returned in the
// same form, so that dL = Re(conj(g_z) dz).
//
//   k_sub_count,     the binned visibilities regrouped by (plane, sub-kernel fv, fu), each
//   k_sub_scatter    with its cell and g, s g (s = -1 for w < 0)
//   k_grad_taps      per (plane, representative sub-kernel): every thread owns one tap of the
//                    quadrant that the x/y mirrors do not cover (as in the resample), and sums
//                    Q = conj(g) G(cell) (w >= 0) or g conj(G(cell)) (w < 0) in registers over
//                    the visibilities of the (up to four) mirror sub-kernels at the tap's
//                    mirror positions -- all at the same radius -- then scatters the sum onto
//                    the radial line through the resample interpolation weights (d/dC_k gets
//                    b Q, d/dC_k+1 gets a Q, the spline second derivatives the cubic weights),
//                    accumulated per block in shared memory and flushed once
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
constexpr int GG_M = 128, GG_N = 128, GG_K = 32;
}  // namespace

// ---- visibilities regrouped by (plane, sub-kernel): key = p os^2 + fv os + fu ----------
__global__ void k_sub_count(const int* __restrict__ n_valid, const int4* __restrict__ srec, int os,
                            int* __restrict__ count2) {
    const int n = *n_valid;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int4 r4 = srec[r];
        atomicAdd(count2 + r4.z * os * os + ((r4.y >> 8) & 0xff) * os + (r4.y & 0xff), 1);
    }
}

__global__ void k_sub_scatter(const int* __restrict__ n_valid, const int4* __restrict__ srec,
                              const float2* __restrict__ gvis, int os, const int* __restrict__ start2,
                              int* __restrict__ cursor2, int* __restrict__ uv2, float4* __restrict__ g4) {
    const int n = *n_valid;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int4 r4 = srec[r];
        const int key = r4.z * os * os + ((r4.y >> 8) & 0xff) * os + (r4.y & 0xff);
        const int pos = start2[key] + atomicAdd(cursor2 + key, 1);
        const float2 g = gvis[r4.w];
        const float sg = ((r4.y >> 16) & 1) ? -1.0f : 1.0f;
        uv2[pos] = r4.x;
        g4[pos] = make_float4(g.x, g.y, sg * g.x, sg * g.y);
    }
}

// Q of one visibility at the grid cell G: conj(g) G for w >= 0, g conj(G) for w < 0, with
// gg = (g, s g): Re Q = g.x G.x + g.y G.y, Im Q = s (g.x G.y - g.y G.x).
__device__ __forceinline__ void q_add(float4 gg, float2 G, float& qr, float& qi) {
    qr = fmaf(gg.x, G.x, fmaf(gg.y, G.y, qr));
    qi = fmaf(gg.z, G.y, fmaf(-gg.w, G.x, qi));
}

// Sum of Q over the visibilities [vb, ve) of one sub-kernel at one footprint position (column
// ca, row ra): TAP_UNROLL visibilities per pass, all their grid loads issued before the sums
// (the loads come from L2 and their latency bounds the kernel).
constexpr int TAP_UNROLL = 8;
__device__ __forceinline__ void tap_sum1(int vb, int ve, int N, int S, const int* __restrict__ uv2,
                                         const float4* __restrict__ g4, const float2* __restrict__ grid, int ca,
                                         int ra, float& qr, float& qi) {
    const int64_t o = (int64_t)(ra - S) * N + (ca - S);
    int v = vb;
    for (; v + TAP_UNROLL <= ve; v += TAP_UNROLL) {
        float2 G[TAP_UNROLL];
#pragma unroll
        for (int i = 0; i < TAP_UNROLL; ++i) {
            const int u = uv2[v + i];
            G[i] = grid[(int64_t)((u >> 16) & 0xffff) * N + (u & 0xffff) + o];
        }
#pragma unroll
        for (int i = 0; i < TAP_UNROLL; ++i) q_add(g4[v + i], G[i], qr, qi);
    }
    for (; v < ve; ++v) {
        const int u = uv2[v];
        q_add(g4[v], grid[(int64_t)((u >> 16) & 0xffff) * N + (u & 0xffff) + o], qr, qi);
    }
}

// Sum of Q over the visibilities [vb, ve) of one sub-kernel at up to two columns (ca, and cb
// when two_c) and two rows (ra, and rb when two_r) of the footprint.  Two visibilities per
// pass, all their grid loads issued before the sums (the loads come from L2).
__device__ __forceinline__ void tap_sum(int vb, int ve, bool on, int N, int S, const int* __restrict__ uv2,
                                        const float4* __restrict__ g4, const float2* __restrict__ grid,
                                        int ca, int cb, bool two_c, int ra, int rb, bool two_r,
                                        float& qr, float& qi) {
    if (!on) return;
    if (!two_c && !two_r) {
        tap_sum1(vb, ve, N, S, uv2, g4, grid, ca, ra, qr, qi);
        return;
    }
    const int64_t o_aa = (int64_t)ra * N + ca, o_ab = (int64_t)ra * N + cb;
    const int64_t o_ba = (int64_t)rb * N + ca, o_bb = (int64_t)rb * N + cb;
    const float2 zero = make_float2(0.0f, 0.0f);
    int v = vb;
    for (; v + 1 < ve; v += 2) {
        const int u0 = uv2[v], u1 = uv2[v + 1];
        const float4 h0 = g4[v], h1 = g4[v + 1];
        const float2* p0 = grid + (int64_t)(((u0 >> 16) & 0xffff) - S) * N + ((u0 & 0xffff) - S);
        const float2* p1 = grid + (int64_t)(((u1 >> 16) & 0xffff) - S) * N + ((u1 & 0xffff) - S);
        const float2 a0 = p0[o_aa], a1 = p1[o_aa];
        const float2 b0 = two_c ? p0[o_ab] : zero, b1 = two_c ? p1[o_ab] : zero;
        const float2 c0 = two_r ? p0[o_ba] : zero, c1 = two_r ? p1[o_ba] : zero;
        const float2 d0 = (two_r && two_c) ? p0[o_bb] : zero, d1 = (two_r && two_c) ? p1[o_bb] : zero;
        q_add(h0, a0, qr, qi);
        q_add(h1, a1, qr, qi);
        q_add(h0, b0, qr, qi);
        q_add(h1, b1, qr, qi);
        q_add(h0, c0, qr, qi);
        q_add(h1, c1, qr, qi);
        q_add(h0, d0, qr, qi);
        q_add(h1, d1, qr, qi);
    }
    if (v < ve) {
        const int u0 = uv2[v];
        const float4 h0 = g4[v];
        const float2* p0 = grid + (int64_t)(((u0 >> 16) & 0xffff) - S) * N + ((u0 & 0xffff) - S);
        q_add(h0, p0[o_aa], qr, qi);
        if (two_c) q_add(h0, p0[o_ab], qr, qi);
        if (two_r) q_add(h0, p0[o_ba], qr, qi);
        if (two_r && two_c) q_add(h0, p0[o_bb], qr, qi);
    }
}

template <bool CUBIC>
__global__ void __launch_bounds__(256) k_grad_taps(int N, int os, int s_max, int K, int nrep, int n_items,
                                                   const int32_t* __restrict__ support,
                                                   const int* __restrict__ start2, const int* __restrict__ uv2,
                                                   const float4* __restrict__ g4, const float2* __restrict__ grid,
                                                   float2* __restrict__ gC, float2* __restrict__ gM) {
    extern __shared__ float2 acc[];    // [ku] d/dC, then [ku] d/dM
    const int item = n_items - 1 - (int)blockIdx.x;   // largest supports first
    const int p = item / nrep;
    const int rep = item - p * nrep;
    const int h = os / 2;
    const int fv = rep / (h + 1), fu = rep - fv * (h + 1);
    const int S = min(max(support[p], 1), s_max);
    const int W = 2 * S + 1;
    const int lim = os * S, lim2 = lim * lim;
    const int ku = min(K, lim + 2);
    for (int k = threadIdx.x; k < (CUBIC ? 2 : 1) * ku; k += blockDim.x) acc[k] = make_float2(0.0f, 0.0f);
    // the quadrant and the mirror maps of the resample
    const int fu2 = fu ? os - fu : 0, fv2 = fv ? os - fv : 0;
    const bool xself = (fu2 == fu), yself = (fv2 == fv);
    const int nx = xself ? S + 1 : W, ny = yself ? S + 1 : W;
    const int cx = fu ? W : W - 1, cy = fv ? W : W - 1;
    const int os2 = os * os;
    const int* s00 = start2 + p * os2 + fv * os + fu;
    const int* s10 = start2 + p * os2 + fv * os + fu2;
    const int* s01 = start2 + p * os2 + fv2 * os + fu;
    const int* s11 = start2 + p * os2 + fv2 * os + fu2;
    const int v00 = s00[0], e00 = s00[1], v10 = s10[0], e10 = s10[1];
    const int v01 = s01[0], e01 = s01[1], v11 = s11[0], e11 = s11[1];
    __syncthreads();
    const int n_eval = nx * ny;
    for (int t0 = 0; t0 < n_eval; t0 += blockDim.x) {
        const int t = t0 + (int)threadIdx.x;
        const int jy = t / nx, jx = t - (t / nx) * nx;
        const int dx = os * (jx - S) - fu, dy = os * (jy - S) - fv;
        const int q = dx * dx + dy * dy;
        const bool on = (t < n_eval) && (q <= lim2);
        const int mj = (jx == 0 && fu) ? 0 : cx - jx;
        const int mjy = (jy == 0 && fv) ? 0 : cy - jy;
        // a sub-kernel that is its own mirror holds the tap at both positions (once if equal)
        const bool x2 = xself && mj != jx, y2 = yself && mjy != jy;
        float qr = 0.0f, qi = 0.0f;
        tap_sum(v00, e00, on, N, S, uv2, g4, grid, jx, mj, x2, jy, mjy, y2, qr, qi);
        if (!xself) tap_sum(v10, e10, on, N, S, uv2, g4, grid, mj, mj, false, jy, mjy, y2, qr, qi);
        if (!yself) tap_sum(v01, e01, on, N, S, uv2, g4, grid, jx, mj, x2, mjy, mjy, false, qr, qi);
        if (!xself && !yself) tap_sum(v11, e11, on, N, S, uv2, g4, grid, mj, mj, false, mjy, mjy, false, qr, qi);
        if (on && (qr != 0.0f || qi != 0.0f)) {
            // the resample's interpolation interval and weights at this radius
            int k;
            float a;
            tap_interval(q, k, a);
            const float b = 1.0f - a;
            atomicAdd(&acc[k].x, b * qr);
            atomicAdd(&acc[k].y, b * qi);
            atomicAdd(&acc[k + 1].x, a * qr);
            atomicAdd(&acc[k + 1].y, a * qi);
            if (CUBIC) {
                const float cb = (b * b - 1.0f) * b * (1.0f / 6.0f);
                const float ca = (a * a - 1.0f) * a * (1.0f / 6.0f);
                atomicAdd(&acc[ku + k].x, cb * qr);
                atomicAdd(&acc[ku + k].y, cb * qi);
                atomicAdd(&acc[ku + k + 1].x, ca * qr);
                atomicAdd(&acc[ku + k + 1].y, ca * qi);
            }
        }
    }
    __syncthreads();
    float2* dC = gC + (int64_t)p * K;
    float2* dM = gM + (int64_t)p * K;
    for (int k = threadIdx.x; k < ku; k += blockDim.x) {
        const float2 c = acc[k];
        if (c.x != 0.0f || c.y != 0.0f) atomicAdd(dC + k, c);
        if (CUBIC) {
            const float2 m = acc[ku + k];
            if (m.x != 0.0f || m.y != 0.0f) atomicAdd(dM + k, m);
        }
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
size_t carve_grad(const Geom& g, int P, int64_t V, void* ws, size_t bytes, GradWork* out) {
    Carver c(ws, bytes);
    GradWork w;
    const int64_t nb2 = (int64_t)P * g.os * g.os;
    w.count2 = c.take<int>((size_t)nb2 + 1);
    w.cursor2 = c.take<int>((size_t)nb2 + 1);
    w.uv2 = c.take<int>((size_t)(V > 0 ? V : 1));
    w.g4 = c.take<float4>((size_t)(V > 0 ? V : 1));
    w.scan_tmp = c.take<int>(scan_tmp_ints(nb2 + 1));
    if (out) *out = w;
    return (size_t)round_up((int64_t)c.off, 256);
}

int grad_radial_run(const Geom& g, const wp_wkernels* kern, const GridWork& w, const GradWork& gw,
                    const float2* gvis, const float2* grid, float2* gC, float2* gM, cudaStream_t st) {
    const int P = kern->P;
    const bool cubic = (g.interp == WP_INTERP_CUBIC);
    WP_CUDA(cudaMemsetAsync(gC, 0, sizeof(float2) * (size_t)P * g.k_out, st));
    if (cubic) WP_CUDA(cudaMemsetAsync(gM, 0, sizeof(float2) * (size_t)P * g.k_out, st));
    const int64_t nb2 = (int64_t)P * g.os * g.os;
    WP_CUDA(cudaMemsetAsync(gw.count2, 0, sizeof(int) * (size_t)(nb2 + 1), st));
    WP_CUDA(cudaMemsetAsync(gw.cursor2, 0, sizeof(int) * (size_t)(nb2 + 1), st));
    int dev = 0, sms = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int* n_valid = w.count + w.nbins;   // binned (not dropped) visibilities
    k_sub_count<<<sms * 4, 256, 0, st>>>(n_valid, w.srec, g.os, gw.count2);
    WP_LAUNCH_CHECK("k_sub_count");
    int rc = exclusive_scan_i32(gw.count2, gw.count2, nb2 + 1, gw.scan_tmp, st);
    if (rc) return rc;
    k_sub_scatter<<<sms * 4, 256, 0, st>>>(n_valid, w.srec, gvis, g.os, gw.count2, gw.cursor2, gw.uv2, gw.g4);
    WP_LAUNCH_CHECK("k_sub_scatter");
    const int h = g.os / 2;
    const int nrep = (h + 1) * (h + 1);
    const int n_items = P * nrep;
    const int ku = g.os * g.s_max + 2 < g.k_out ? g.os * g.s_max + 2 : g.k_out;
    const size_t smem = (size_t)(cubic ? 2 : 1) * ku * sizeof(float2);
    if (cubic) {
        if (smem > 48 * 1024)
            WP_CUDA(cudaFuncSetAttribute(k_grad_taps<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_grad_taps<true><<<n_items, 256, smem, st>>>(g.N, g.os, g.s_max, g.k_out, nrep, n_items, w.seff,
                                                      gw.count2, gw.uv2, gw.g4, grid, gC, gM);
    } else {
        if (smem > 48 * 1024)
            WP_CUDA(cudaFuncSetAttribute(k_grad_taps<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_grad_taps<false><<<n_items, 256, smem, st>>>(g.N, g.os, g.s_max, g.k_out, nrep, n_items, w.seff,
                                                       gw.count2, gw.uv2, gw.g4, grid, gC, gM);
    }
    WP_LAUNCH_CHECK("k_grad_taps");
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
