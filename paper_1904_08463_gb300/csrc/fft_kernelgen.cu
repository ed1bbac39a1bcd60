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
//
// The projection-slice Hankel route (Section 4.3.1, Alg. 2 steps 4-12) shares the workspace:
// the same image-domain samples are summed over one axis (the projection p(l)), the line is
// zero-padded to L = M os and transformed by a batched 1D cuFFT; its sample k is the v = 0
// slice of the 2D route's transform at uv offset k du / os -- the radial kernel line, which
// then goes through the same truncation, spline and resample as the matrix route.
//   k_ps_nm1       n - 1 at the workspace pixels as float pairs (FP64 once per geometry)
//   k_ps_project   column sums (rows +dy and -dy paired), line zeroed beforehand
//   cuFFT          forward C2C, length L, batched over planes
//   k_ps_extract   radial[p][k] = line[p][k mod L]
#include <cuda_runtime.h>
#include <cufft.h>

#include <map>
#include <mutex>
#include <tuple>

#include "wp_internal.cuh"

namespace wp {

namespace {
std::mutex g_mu;
// (device, L, batch, stream) -> plan: one plan (and work area) per stream, so concurrent
// calls on different streams never share a work area
std::map<std::tuple<int, int, int, uintptr_t>, cufftHandle> g_plans;

int plan_many(int L, int batch, cudaStream_t st, cufftHandle* out) {
    int dev = 0;
    WP_CUDA(cudaGetDevice(&dev));
    auto key = std::make_tuple(dev, L, batch, (uintptr_t)st);
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
    const int S = fit_support(min(max(support[p], 1), s_max), os, offsets, p);
    if (S < 1) return;
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
        int rc = plan_many(L, nb, st, &h);
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

// ---------------------------------------------------------------------------------------
// projection-slice route
// ---------------------------------------------------------------------------------------
namespace {
std::map<std::tuple<int, int, int, uintptr_t>, cufftHandle> g_plans1d;   // (device, L, batch, stream)

int plan_1d(int L, int batch, cudaStream_t st, cufftHandle* out) {
    int dev = 0;
    WP_CUDA(cudaGetDevice(&dev));
    auto key = std::make_tuple(dev, L, batch, (uintptr_t)st);
    auto it = g_plans1d.find(key);
    if (it != g_plans1d.end()) { *out = it->second; return WP_OK; }
    cufftHandle h;
    int n[1] = {L};
    if (cufftPlanMany(&h, 1, n, nullptr, 1, L, nullptr, 1, L, CUFFT_C2C, batch) != CUFFT_SUCCESS) {
        set_last_error("cufftPlanMany", "1D plan creation failed");
        return WP_ERR_CUDA;
    }
    g_plans1d[key] = h;
    *out = h;
    return WP_OK;
}
}  // namespace

void release_ps_plans() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_plans1d) cufftDestroy(kv.second);
    g_plans1d.clear();
}

// n - 1 = -r^2 / (1 + sqrt(1 - r^2)) at the workspace pixels (0 outside the unit circle),
// in FP64, stored as the float pair (nearest float, nearest float to the rest).
__global__ void k_ps_nm1(int M, double dlw, float2* __restrict__ nm1f) {
    const int jx = blockIdx.x * blockDim.x + threadIdx.x, jy = blockIdx.y;
    if (jx >= M) return;
    const double l = (double)(jx - M / 2) * dlw, m = (double)(jy - M / 2) * dlw;
    const double r2 = l * l + m * m;
    const double v = (r2 < 1.0) ? -r2 / (1.0 + sqrt(1.0 - r2)) : 0.0;
    const float hi = (float)v;
    nm1f[(int64_t)jy * M + jx] = make_float2(hi, (float)(v - (double)hi));
}

// Block (column group, plane): PS_COLS workspace columns x PS_ROWG row groups.  The
// workspace value depends on the pixel only through d^2 = dx^2 + dy^2, so rows +dy and -dy
// are equal: a column sum is f(dy = -M/2) + f(0) + 2 sum_{dy = 1}^{M/2 - 1} f(dy).  Each
// thread sums its share of dy >= 1, the row groups are combined in shared memory, and the
// column's sum lands at line index (jx - M/2) mod L (the rest of the line is zeroed
// beforehand).  The workspace value is the 2D route's: taper (linear between its nodes) x
// screen inside the disc r <= r_max (tested on integer offsets), the phase w (n - 1) from
// float pairs (exact high product + cross terms, exact reduction by the nearest integer),
// scaled by (FOV / M)^2 du^2 = 1 / M^2.
constexpr int PS_COLS = 32, PS_ROWG = 8;

__device__ __forceinline__ float2 ps_value(int M, int R, int jx, int jy, float2 w, const float2* __restrict__ nm1f,
                                           const float* __restrict__ taper) {
    const int h = M / 2;
    const int dx = jx - h, dy = jy - h;
    const int d2 = dx * dx + dy * dy;
    if (d2 > h * h) return make_float2(0.0f, 0.0f);
    float x = 2.0f * (float)R * sqrtf((float)d2) / (float)M - 0.5f;
    x = fminf(fmaxf(x, 0.0f), (float)(R - 1));
    const int i0 = min((int)x, R - 2);
    const float a = x - (float)i0;
    const float t = (1.0f - a) * taper[i0] + a * taper[i0 + 1];
    const float2 n = nm1f[(int64_t)jy * M + jx];
    const float ph = w.x * n.x;
    float pl = fmaf(w.x, n.x, -ph);
    pl = fmaf(w.x, n.y, fmaf(w.y, n.x, pl));
    const float fr = (ph - rintf(ph)) + pl;
    float s, c;
    sincospif(2.0f * fr, &s, &c);
    return make_float2(t * c, t * s);
}

__global__ void __launch_bounds__(PS_COLS * PS_ROWG) k_ps_project(int M, int L, int R, const float2* __restrict__ nm1f,
                                                                 const float* __restrict__ taper,
                                                                 const double* __restrict__ w_planes,
                                                                 float2* __restrict__ X) {
    __shared__ float2 part[PS_ROWG][PS_COLS];
    __shared__ float2 wsplit;
    const int p = blockIdx.y;
    if (threadIdx.x == 0) {
        const double wd = w_planes[p];
        const float hi = (float)wd;
        wsplit = make_float2(hi, (float)(wd - (double)hi));
    }
    __syncthreads();
    const int c = threadIdx.x % PS_COLS, rg = threadIdx.x / PS_COLS;
    const int jx = blockIdx.x * PS_COLS + c;
    const int h = M / 2;
    const float2 w = wsplit;
    float sr = 0.0f, si = 0.0f;
    if (jx < M) {
        for (int dy = 1 + rg; dy < h; dy += PS_ROWG) {     // rows h + dy (and their mirrors h - dy)
            const float2 v = ps_value(M, R, jx, h + dy, w, nm1f, taper);
            sr += v.x;
            si += v.y;
        }
        sr *= 2.0f;
        si *= 2.0f;
        if (rg == 0) {                                     // the unpaired rows dy = 0 and dy = -M/2
            const float2 v0 = ps_value(M, R, jx, h, w, nm1f, taper);
            const float2 v1 = ps_value(M, R, jx, 0, w, nm1f, taper);
            sr += v0.x + v1.x;
            si += v0.y + v1.y;
        }
    }
    part[rg][c] = make_float2(sr, si);
    __syncthreads();
    if (rg == 0 && jx < M) {
        float2 acc = part[0][c];
        for (int q = 1; q < PS_ROWG; ++q) {
            acc.x += part[q][c].x;
            acc.y += part[q][c].y;
        }
        const float inv_m2 = 1.0f / ((float)M * (float)M);
        X[(int64_t)p * L + (jx - h + L) % L] = make_float2(acc.x * inv_m2, acc.y * inv_m2);
    }
}

__global__ void k_ps_extract(int K, int L, const float2* __restrict__ Y, float2* __restrict__ radial) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
    if (k >= K) return;
    radial[(int64_t)p * K + k] = Y[(int64_t)p * L + (k % L)];
}

int kg_ps_prepare(const Geom& g, const KgWork& w, cudaStream_t st) {
    const int M = g.fft_m;
    k_ps_nm1<<<dim3((M + 127) / 128, M), 128, 0, st>>>(M, (double)g.N * g.dl / M, w.ps_nm1);
    WP_LAUNCH_CHECK("k_ps_nm1");
    return WP_OK;
}

int kg_projslice(const Geom& g, const KgWork& w, const float* taper, const double* w_planes, int P,
                 float2* radial, cudaStream_t st) {
    const int M = g.fft_m;
    const int L = M * g.os;
    WP_CUDA(cudaMemsetAsync(w.ps_x, 0, (size_t)P * L * sizeof(float2), st));
    k_ps_project<<<dim3((M + PS_COLS - 1) / PS_COLS, P), PS_COLS * PS_ROWG, 0, st>>>(M, L, g.R, w.ps_nm1, taper,
                                                                                   w_planes, w.ps_x);
    WP_LAUNCH_CHECK("k_ps_project");
    {
        std::lock_guard<std::mutex> lk(g_mu);
        cufftHandle h;
        int rc = plan_1d(L, P, st, &h);
        if (rc) return rc;
        if (cufftSetStream(h, st) != CUFFT_SUCCESS ||
            cufftExecC2C(h, reinterpret_cast<cufftComplex*>(w.ps_x), reinterpret_cast<cufftComplex*>(w.ps_x),
                         CUFFT_FORWARD) != CUFFT_SUCCESS) {
            set_last_error("cufftExecC2C", "batched 1D transform failed");
            return WP_ERR_CUDA;
        }
    }
    k_ps_extract<<<dim3((g.k_out + 255) / 256, P), 256, 0, st>>>(g.k_out, L, w.ps_x, radial);
    WP_LAUNCH_CHECK("k_ps_extract");
    return WP_OK;
}

}  // namespace wp
