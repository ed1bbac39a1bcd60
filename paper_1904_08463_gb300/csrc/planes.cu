// w-plane values (Alg. 1 / Alg. 2 steps 1-3 of the paper): sort the visibilities' |w|,
// cut the sorted list into P equal-count chunks (the first V mod P chunks one longer) and
// take each chunk's mean -- the paper's default of average w per plane.  The sort is the
// library's own radix sort (sort.cu) of the float bit patterns (non-negative floats order like
// their bits); the chunk means are FP64 sums, one block per chunk.  Non-finite |w| (bit patterns from
// 0x7F800000 up) sort last and take no part: the chunks cut the finite values only, and a
// chunk left empty (fewer finite values than planes) takes the largest finite |w| (0 if none),
// so the plane values stay ascending; binning drops such visibilities.
#include <cuda_runtime.h>

#include "wp_internal.cuh"

namespace wp {

__global__ void k_abs_w_keys(int64_t V, const float* __restrict__ uvw, unsigned* __restrict__ keys) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < V) keys[k] = __float_as_uint(fabsf(uvw[3 * k + 2]));
}

// number of finite |w| in the ascending keys (one thread: a binary search)
__global__ void k_finite_count(int64_t V, const unsigned* __restrict__ sorted, int64_t* __restrict__ nf) {
    int64_t lo = 0, hi = V;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (sorted[mid] < 0x7F800000u) lo = mid + 1; else hi = mid;
    }
    *nf = lo;
}

__global__ void __launch_bounds__(256) k_chunk_means(int P, const unsigned* __restrict__ sorted,
                                                     const int64_t* __restrict__ nf, double* __restrict__ out) {
    __shared__ double red[8];
    const int c = blockIdx.x;
    const int64_t V = *nf;
    const int64_t q = V / P, r = V % P;
    const int64_t beg = (int64_t)c * q + (c < r ? c : r);
    const int64_t n = q + (c < r ? 1 : 0);
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)__uint_as_float(sorted[beg + i]);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[c] = n > 0 ? t / (double)n : (V > 0 ? (double)__uint_as_float(sorted[V - 1]) : 0.0);
    }
}

size_t plane_values_workspace_bytes(int64_t V) {
    Carver c(nullptr, 0);
    c.take<unsigned>((size_t)V);
    c.take<unsigned>((size_t)V);
    c.take<int64_t>(1);
    c.take<int>(radix_sort_hist_ints(V));
    c.take<int>(scan_tmp_ints((int64_t)radix_sort_hist_ints(V)));
    return (size_t)round_up((int64_t)c.off, 256);
}

int plane_values(const float* uvw, int64_t V, int P, void* ws, size_t bytes, double* out, cudaStream_t st) {
    Carver c(ws, bytes);
    unsigned* keys = c.take<unsigned>((size_t)V);
    unsigned* alt = c.take<unsigned>((size_t)V);
    int64_t* nf = c.take<int64_t>(1);
    int* hist = c.take<int>(radix_sort_hist_ints(V));
    int* stmp = c.take<int>(scan_tmp_ints((int64_t)radix_sort_hist_ints(V)));
    k_abs_w_keys<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(V, uvw, keys);
    WP_LAUNCH_CHECK("k_abs_w_keys");
    bool in_alt = false;
    // |w| has a clear sign bit: bits 0..30 order the keys (four 8-bit passes)
    int rc = radix_sort<uint32_t>(keys, nullptr, alt, nullptr, V, 31, hist, stmp, st, &in_alt);
    if (rc) return rc;
    const unsigned* sorted = in_alt ? alt : keys;
    k_finite_count<<<1, 1, 0, st>>>(V, sorted, nf);
    WP_LAUNCH_CHECK("k_finite_count");
    k_chunk_means<<<P, 256, 0, st>>>(P, sorted, nf, out);
    WP_LAUNCH_CHECK("k_chunk_means");
    return WP_OK;
}

}  // namespace wp
