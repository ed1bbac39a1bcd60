// Measurement helper with no counterpart in the paper: the FP32 FMA rate of the device, the
// denominator of the gridder's ALU roofline, measured on the GPU that runs the library instead of
// taken from a nominal figure (SMs x FP32 lanes x 2 x clock).
//
// Every thread runs eight independent FMA chains held in registers (no memory traffic inside the
// timed loop); the caller times the launch with CUDA events and divides the FLOP count the call
// reports by the elapsed time.
#include <cuda_runtime.h>

#include <cstdint>

#include "wp_internal.cuh"

namespace wp {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

__global__ void __launch_bounds__(PROBE_THREADS) k_fma_rate(int iters, float* __restrict__ sink) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = (float)(threadIdx.x + c);
    const float b = 0.999f, d = 0.001f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = fmaf(a[c], b, d);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
    if (s == 12345.0f) sink[0] = s;   // keeps the chains live; never true for these inputs
}

}  // namespace wp

using namespace wp;

extern "C" int wp_probe_fp32_fma(int32_t iters, int32_t blocks_per_sm, float* sink, double* flops_out,
                                 void* stream) {
    if (!sink || !flops_out) return WP_ERR_NULL;
    if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64) return WP_ERR_SIZE;
    int rc = check_device_public();
    if (rc) return rc;
    int dev = 0, sms = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * blocks_per_sm;
    k_fma_rate<<<blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(iters, sink);
    WP_LAUNCH_CHECK("k_fma_rate");
    *flops_out = 2.0 * PROBE_CHAINS * PROBE_UNROLL * (double)iters * (double)blocks * PROBE_THREADS;
    return WP_OK;
}

namespace wp {

constexpr int PROBE_TAP_ROWS = 10;

// Each warp, per step: a pseudo-random base in [0, span) of the buffer, then PROBE_TAP_ROWS rows
// base + r W + lane -- one 8-byte load per lane per row, the shape of the slot gridder's tap loads
// (rows of one sub-kernel at a footprint offset that is any multiple of 8 bytes).  Every index is
// below span + (PROBE_TAP_ROWS - 1) W + 32, which the host checks against the buffer.
__global__ void __launch_bounds__(PROBE_THREADS) k_l2_taps(const float2* __restrict__ buf, uint32_t span, int W,
                                                           int steps, float* __restrict__ sink) {
    const int lane = threadIdx.x & 31;
    uint32_t h = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2654435761u + 12345u;
    float sx = 0.0f, sy = 0.0f;
    for (int s = 0; s < steps; ++s) {
        h = h * 1664525u + 1013904223u;
        const size_t base = (size_t)(h % span);
        float2 v[PROBE_TAP_ROWS];
#pragma unroll
        for (int r = 0; r < PROBE_TAP_ROWS; ++r) v[r] = __ldg(buf + base + (size_t)r * W + lane);
#pragma unroll
        for (int r = 0; r < PROBE_TAP_ROWS; ++r) {
            sx += v[r].x;
            sy += v[r].y;
        }
    }
    if (sx == 12345.0f && sy == 54321.0f) sink[0] = sx;   // keeps the loads live; never true here
}

}  // namespace wp

extern "C" int wp_probe_l2_taps(const void* buf, int64_t n_elems, int32_t W, int32_t steps, int32_t blocks_per_sm,
                                float* sink, double* bytes_out, void* stream) {
    if (!buf || !sink || !bytes_out) return WP_ERR_NULL;
    if (W < 1 || W > 4096 || steps < 1 || blocks_per_sm < 1 || blocks_per_sm > 64) return WP_ERR_SIZE;
    const int64_t reach = (int64_t)(PROBE_TAP_ROWS - 1) * W + 32;
    if (n_elems <= reach || n_elems - reach > (int64_t)0xffffffffLL) return WP_ERR_SIZE;
    if (reinterpret_cast<uintptr_t>(buf) % 8) return WP_ERR_SIZE;
    int rc = check_device_public();
    if (rc) return rc;
    int dev = 0, sms = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * blocks_per_sm;
    k_l2_taps<<<blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(static_cast<const float2*>(buf),
                                                                  (uint32_t)(n_elems - reach), W, steps, sink);
    WP_LAUNCH_CHECK("k_l2_taps");
    *bytes_out = 8.0 * PROBE_TAP_ROWS * 32.0 * (double)steps * (double)blocks * (PROBE_THREADS / 32);
    return WP_OK;
}
