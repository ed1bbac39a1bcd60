// Grid <-> image (Section 3 of the paper: inverse transform of the grid, then division by
// the transform of the anti-aliasing function; Section 6: the Hankel-route image is valid
// inside the circle whose diameter is the image size).
//
// The centred transform  sum_u g[u] exp(+2 pi j (u - N/2)(l - N/2) / N)  is an ordinary
// unnormalised inverse DFT read at (l + N/2) mod N and multiplied by (-1)^l (per axis;
// the constant phase of the two axes cancels for even N), so the fftshifts are folded
// into the correction kernels instead of being separate passes.  The DFT itself is a
// cuFFT C2C call (the hand-written inverse transform is out of scope).
#include <cuda_runtime.h>
#include <cufft.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "wp_internal.cuh"

namespace wp {

namespace {
std::mutex g_fft_mu;
// (device, N, stream) -> plan: a plan's work area may serve one stream at a time, and
// independent problems run their transforms concurrently on separate streams (also inside a
// captured graph), so each stream has its own plan.
std::map<std::tuple<int, int, uintptr_t>, cufftHandle> g_fft_plans;

int get_plan(int N, cudaStream_t st, cufftHandle* out) {
    int dev = 0;
    WP_CUDA(cudaGetDevice(&dev));
    auto key = std::make_tuple(dev, N, (uintptr_t)st);
    auto it = g_fft_plans.find(key);
    if (it != g_fft_plans.end()) {
        *out = it->second;
        return WP_OK;
    }
    cufftHandle h;
    cufftResult r = cufftPlan2d(&h, N, N, CUFFT_C2C);
    if (r != CUFFT_SUCCESS) {
        set_last_error("cufftPlan2d", "plan creation failed");
        return WP_ERR_CUDA;
    }
    g_fft_plans[key] = h;
    *out = h;
    return WP_OK;
}

int exec_fft(int N, float2* data, int direction, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_fft_mu);
    cufftHandle h;
    int rc = get_plan(N, st, &h);
    if (rc) return rc;
    if (cufftSetStream(h, st) != CUFFT_SUCCESS) {
        set_last_error("cufftSetStream", "failed");
        return WP_ERR_CUDA;
    }
    cufftResult r = cufftExecC2C(h, reinterpret_cast<cufftComplex*>(data),
                                 reinterpret_cast<cufftComplex*>(data), direction);
    if (r != CUFFT_SUCCESS) {
        set_last_error("cufftExecC2C", "execution failed");
        return WP_ERR_CUDA;
    }
    return WP_OK;
}
}  // namespace

void release_fft_plans() {
    std::lock_guard<std::mutex> lk(g_fft_mu);
    for (auto& kv : g_fft_plans) cufftDestroy(kv.second);
    g_fft_plans.clear();
}

// t(r) by linear interpolation between the radial nodes r_i = (i + 1/2) r_max / R, clamped
// at the end nodes; x = r / dr - 1/2 = 2 R d / N - 1/2 for a pixel at distance d (pixels).
__device__ __forceinline__ float taper_at_pixel(const float* __restrict__ taper, int R, int N, int d2) {
    float x = 2.0f * (float)R * sqrtf((float)d2) / (float)N - 0.5f;
    x = fminf(fmaxf(x, 0.0f), (float)(R - 1));
    int i0 = min((int)x, R - 2);
    float a = x - (float)i0;
    return (1.0f - a) * taper[i0] + a * taper[i0 + 1];
}

// inv_wsum is 1 / weight_sum from the host, or, when wsum_dev is set, 1 / wsum_dev[0] read on the
// device (the weight sum wp_grid accumulated in its stats) -- one FP64 division per block, broadcast
// through shared memory; a sum <= 0 (nothing gridded) gives a zero image.
__global__ void k_dirty_correct(int N, int R, const float* __restrict__ taper, float inv_wsum,
                                const double* __restrict__ wsum_dev, const float2* __restrict__ F,
                                float* __restrict__ image) {
    __shared__ float s_inv;
    if (wsum_dev) {
        if (threadIdx.x == 0) {
            const double s = wsum_dev[0];
            s_inv = (s > 0.0) ? (float)(1.0 / s) : 0.0f;
        }
        __syncthreads();
        inv_wsum = s_inv;
    }
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (l >= N) return;
    int h = N / 2;
    int dl_ = l - h, dm_ = m - h;
    int d2 = dl_ * dl_ + dm_ * dm_;
    float out = 0.0f;
    if (d2 <= h * h) {
        float v = F[(int64_t)((m + h) % N) * N + ((l + h) % N)].x;
        if ((l + m) & 1) v = -v;
        out = v * inv_wsum / taper_at_pixel(taper, R, N, d2);
    }
    image[(int64_t)m * N + l] = out;
}

__global__ void k_image_pre(int N, int R, const float* __restrict__ taper, float inv_wsum,
                            const float* __restrict__ image, float2* __restrict__ G) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (l >= N) return;
    int h = N / 2;
    int dl_ = l - h, dm_ = m - h;
    int d2 = dl_ * dl_ + dm_ * dm_;
    float v = 0.0f;
    if (d2 <= h * h) {
        v = image[(int64_t)m * N + l] * inv_wsum / taper_at_pixel(taper, R, N, d2);
        if ((l + m) & 1) v = -v;
    }
    G[(int64_t)m * N + l] = make_float2(v, 0.0f);
}

__global__ void k_checker(int N, float2* __restrict__ G) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int v = blockIdx.y;
    if (u >= N) return;
    if ((u + v) & 1) {
        float2 x = G[(int64_t)v * N + u];
        G[(int64_t)v * N + u] = make_float2(-x.x, -x.y);
    }
}

int image_dirty(const Geom& g, const float* taper, float2* grid, double wsum, const double* wsum_dev,
                float* image, cudaStream_t st) {
    int rc = exec_fft(g.N, grid, CUFFT_INVERSE, st);
    if (rc) return rc;
    dim3 blk(256), grd((g.N + 255) / 256, g.N);
    const float inv = wsum_dev ? 0.0f : (float)(1.0 / wsum);
    k_dirty_correct<<<grd, blk, 0, st>>>(g.N, g.R, taper, inv, wsum_dev, grid, image);
    WP_LAUNCH_CHECK("k_dirty_correct");
    return WP_OK;
}

int image_to_grid(const Geom& g, const float* taper, const float* image, double wsum, float2* grid,
                  cudaStream_t st) {
    dim3 blk(256), grd((g.N + 255) / 256, g.N);
    k_image_pre<<<grd, blk, 0, st>>>(g.N, g.R, taper, (float)(1.0 / wsum), image, grid);
    WP_LAUNCH_CHECK("k_image_pre");
    int rc = exec_fft(g.N, grid, CUFFT_FORWARD, st);
    if (rc) return rc;
    k_checker<<<grd, blk, 0, st>>>(g.N, grid);
    WP_LAUNCH_CHECK("k_checker");
    return WP_OK;
}

int image_adjoint(const Geom& g, const float* taper, const float* image, float2* grid_g, double wsum,
                  float* grad_image, float* grad_taper, cudaStream_t st) {
    int rc = exec_fft(g.N, grid_g, CUFFT_INVERSE, st);
    if (rc) return rc;
    return launch_image_adjoint(g, taper, image, grid_g, wsum, grad_image, grad_taper, st);
}

}  // namespace wp
