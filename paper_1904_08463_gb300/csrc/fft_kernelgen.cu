// Standard w-projection kernel generation by 2D FFT (Alg. 1 steps 4-11 of the paper, with
// the workspace undersampling of Section 4.2) -- the comparator of the Hankel route.
//
// Per plane: the image-domain product taper x w-screen is sampled on an M x M workspace
// spanning the whole field of view (M = power of two >= 2 S_max + 1, pixel FOV / M),
// zero-padded to L = M os, transformed with a batched cuFFT C2C, and the oversampled
// kernel cache is read off the fine grid: fine sample a sits at uv offset a du / os, and
// tap (jx, jy) of sub-kernel (fu, fv) is the sample at (os (jx - S) - fu, os (jy - S) - fv).
// The image-domain function is zero outside the circle of radius r_max (the same disc the
// Hankel route integrates over) and taps beyond the support radius are zeroed when
// `circular` is set, so both routes compute the same kernels.
//   k_fft_fill     writes the M x M workspace samples into the zeroed padded buffer
//                  (FP64 phase from a per-pixel n - 1 table, reduced to [-1/2, 1/2] cycles)
//   cuFFT          forward C2C, L x L, batched over planes
//   k_fft_extract  one thread per fine-grid sample of the plane's footprint: reads the FFT
//                  output row-contiguously, writes each tap to its sub-kernel (32-byte runs)
#include <cuda_runtime.h>
#include <cufft.h>

#include <map>
#include <mutex>
#include <tuple>

#include "wp_internal.cuh"

namespace wp {

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int>, cufftHandle> g_plans;   // (device, L, batch) -> plan

int plan_many(int L, int batch, cufftHandle* out) {
    int dev = 0;
    WP_CUDA(cudaGetDevice(&dev));
    auto key = std::make_tuple(dev, L, batch);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) { *out = it->second; return WP_OK; }
    cufftHandle h;
    int n[2] = {L, L};
    if (cufftPlanMany(&h, 2, n, nullptr, 1, L * L, nullptr, 1, L * L, CUFFT_C2C, batch) != CUFFT_SUCCESS) {
        set_last_error("cufftPlanMany", "plan creation failed");
        return WP_ERR_CUDA;
    }
    g_plans[key] = h;
    *out = h;
    return WP_OK;
}
}  // namespace

void release_fft_kernelgen_plans() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_plans) cufftDestroy(kv.second);
    g_plans.clear();
}

int fft_batch_planes(const Geom& g, int P) {
    const int64_t L = (int64_t)g.fft_m * g.os;
    int64_t b = ((int64_t)1 << 30) / (L * L * 8);
    if (b < 1) b = 1;
    if (b > P) b = P;
    return (int)b;
}

size_t fft_workspace_bytes(const Geom& g, int P) {
    const int64_t L = (int64_t)g.fft_m * g.os;
    const int M = g.fft_m;
    Carver c(nullptr, 0);
    c.take<float2>((size_t)fft_batch_planes(g, P) * L * L);
    c.take<double>((size_t)M * M);
    return (size_t)round_up((int64_t)c.off, 256);
}

// n - 1 at the workspace pixels, FP64 without cancellation, and 0 outside the circle
// (which the fill kernel tests exactly on integers).
__global__ void k_fft_nm1(int M, double dlw, double* __restrict__ nm1) {
    const int jx = blockIdx.x * blockDim.x + threadIdx.x, jy = blockIdx.y;
    if (jx >= M) return;
    const double l = (double)(jx - M / 2) * dlw, m = (double)(jy - M / 2) * dlw;
    const double r2 = l * l + m * m;
    nm1[(int64_t)jy * M + jx] = (r2 < 1.0) ? -r2 / (1.0 + sqrt(1.0 - r2)) : 0.0;
}

__global__ void k_fft_fill(int M, int L, int R, int p0, int nb, const double* __restrict__ nm1,
                           const float* __restrict__ taper, const double* __restrict__ w_planes,
                           float2* __restrict__ X) {
    const int jx = blockIdx.x * blockDim.x + threadIdx.x, jy = blockIdx.y, b = blockIdx.z;
    if (jx >= M || b >= nb) return;
    const int dx = jx - M / 2, dy = jy - M / 2;
    const int d2 = dx * dx + dy * dy;
    float2 v = make_float2(0.0f, 0.0f);
    if (d2 <= (M / 2) * (M / 2)) {              // inside the disc r <= r_max (exact)
        // taper between its nodes r_i = (i + 1/2) r_max / R: x = 2 R d / M - 1/2
        float x = 2.0f * (float)R * sqrtf((float)d2) / (float)M - 0.5f;
        x = fminf(fmaxf(x, 0.0f), (float)(R - 1));
        const int i0 = min((int)x, R - 2);
        const float a = x - (float)i0;
        const float t = (1.0f - a) * taper[i0] + a * taper[i0 + 1];
        const double cyc = w_planes[p0 + b] * nm1[(int64_t)jy * M + jx];
        const double fr = cyc - rint(cyc);
        float s, c;
        sincospif((float)(2.0 * fr), &s, &c);
        // (FOV / M)^2 du^2 = 1 / M^2 carries the transform's scale and the tap normalisation
        const float sc = t / ((float)M * (float)M);
        v = make_float2(sc * c, sc * s);
    }
    const int ay = (dy + L) % L, ax = (dx + L) % L;
    X[(int64_t)b * L * L + (int64_t)ay * L + ax] = v;
}

__global__ void __launch_bounds__(256) k_fft_extract(int L, int os, int s_max, int p0, int circular,
                                                     const int32_t* __restrict__ support,
                                                     const int64_t* __restrict__ offsets,
                                                     const float2* __restrict__ Y, float2* __restrict__ cache) {
    const int b = blockIdx.z;
    const int p = p0 + b;
    const int S = min(max(support[p], 1), s_max);
    const int W = 2 * S + 1;
    const int span = os * W;                        // fine samples per axis of the footprint
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y;
    if (ix >= span || iy >= span) return;
    // fine offsets a in [-os S - os + 1, os S]
    const int ax = ix - os * S - os + 1, ay = iy - os * S - os + 1;
    const int fu = ((-ax) % os + os) % os, fv = ((-ay) % os + os) % os;
    const int jx = (ax + fu) / os + S, jy = (ay + fv) / os + S;
    const float2* src = Y + (int64_t)b * L * L;
    float2 v = src[(int64_t)((ay + L) % L) * L + ((ax + L) % L)];
    if (circular) {
        const int lim = os * S;
        if (ax * ax + ay * ay > lim * lim) v = make_float2(0.0f, 0.0f);
    }
    cache[offsets[p] + ((int64_t)(fv * os + fu) * W + jy) * W + jx] = v;
}

int fft_wkernels(const Geom& g, const float* taper, const double* w_planes, int P, const int32_t* support,
                 const int64_t* offsets, int circular, void* ws, size_t ws_bytes, float2* cache,
                 cudaStream_t st) {
    const int M = g.fft_m;
    const int L = M * g.os;
    const int B = fft_batch_planes(g, P);
    Carver c(ws, ws_bytes);
    float2* X = c.take<float2>((size_t)B * L * L);
    double* nm1 = c.take<double>((size_t)M * M);
    k_fft_nm1<<<dim3((M + 127) / 128, M), 128, 0, st>>>(M, (double)g.N * g.dl / M, nm1);
    WP_LAUNCH_CHECK("k_fft_nm1");
    std::lock_guard<std::mutex> lk(g_mu);
    for (int p0 = 0; p0 < P; p0 += B) {
        const int nb = (P - p0 < B) ? (P - p0) : B;
        cufftHandle h;
        int rc = plan_many(L, nb, &h);
        if (rc) return rc;
        WP_CUDA(cudaMemsetAsync(X, 0, (size_t)nb * L * L * sizeof(float2), st));
        k_fft_fill<<<dim3((M + 127) / 128, M, nb), 128, 0, st>>>(M, L, g.R, p0, nb, nm1, taper, w_planes, X);
        WP_LAUNCH_CHECK("k_fft_fill");
        if (cufftSetStream(h, st) != CUFFT_SUCCESS ||
            cufftExecC2C(h, reinterpret_cast<cufftComplex*>(X), reinterpret_cast<cufftComplex*>(X),
                         CUFFT_FORWARD) != CUFFT_SUCCESS) {
            set_last_error("cufftExecC2C", "batched forward transform failed");
            return WP_ERR_CUDA;
        }
        const int span_max = g.os * (2 * g.s_max + 1);
        k_fft_extract<<<dim3((span_max + 255) / 256, span_max, nb), 256, 0, st>>>(
            L, g.os, g.s_max, p0, circular, support, offsets, X, cache);
        WP_LAUNCH_CHECK("k_fft_extract");
    }
    return WP_OK;
}

}  // namespace wp
