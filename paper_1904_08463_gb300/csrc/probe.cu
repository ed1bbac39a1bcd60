// Measurement helper with no counterpart in the paper: the FP32 FMA rate of the device, the
// denominator of the gridder's ALU roofline, measured on the GPU that runs the library instead of
// taken from a nominal figure (SMs x FP32 lanes x 2 x clock).
//
// Every thread runs eight independent FMA chains held in registers (no memory traffic inside the
// timed loop); the caller times the launch with CUDA events and divides the FLOP count the call
// reports by the elapsed time.
#include <cuda_runtime.h>

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
