// Gridding without any device allocation by the library or the caller.
//
// wp_grid needs scratch (binned records, bin counts, work items) that the caller normally
// allocates and passes in.  Some callers cannot do that: an imaging pipeline that reserves
// every byte of HBM for its own pools at start-up and forbids later allocations (so that a
// long observation never fragments memory or fails half-way), or a host framework whose
// plug-ins may only use memory it hands them.  wp_grid_static gives those callers the same
// gridding with the scratch taken from one fixed-size array compiled into this library.
#include <cuda_runtime.h>

#include <mutex>

#include "wp_internal.cuh"

namespace wp {
namespace {

// The scratch.  A device holds these bytes from the first wp_grid_static call on it until the
// process exits: the runtime loads this file's module (and with it the array) lazily, when the
// set-up below asks for the array's address -- not when the library is loaded.
constexpr size_t kStaticScratchBytes = (size_t)WP_GRID_STATIC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_grid_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[64] = {};   // device address of g_grid_scratch, per device ordinal

// Once per device, with that device current: the host-side symbol is only a stand-in, the
// device address must come from the runtime.
int scratch_for_current_device(void** out) {
    int dev = 0;
    WP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return WP_ERR_DEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_grid_scratch);
        if (e != cudaSuccess) return cuda_fail("cudaGetSymbolAddress(g_grid_scratch)", e);
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return WP_OK;
}

}  // namespace
}  // namespace wp

using namespace wp;

extern "C" int wp_grid_static(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw,
                              const float* vis, const float* weight, int64_t V, float* grid,
                              double* stats, void* stream) {
    WP_RANGE("wp_grid_static");
    Geom g;
    // wp_grid's own checks (plan, kernels, sizes, device), minus the caller workspace
    int rc = check_grid_args(plan, kernels, uvw, V, nullptr, 0, &g, true, false);
    if (rc) return rc;
    if (!grid || (V > 0 && !vis)) return WP_ERR_NULL;
    const size_t need = carve_grid(g, kernels->P, V, nullptr, 0, nullptr);
    if (need > kStaticScratchBytes) {
        set_last_error("wp_grid_static", "problem needs more scratch than the static array holds "
                                         "(WP_GRID_STATIC_SCRATCH_BYTES); use wp_grid");
        return WP_ERR_SIZE;
    }
    void* scratch = nullptr;
    if ((rc = scratch_for_current_device(&scratch))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    GridWork w;
    carve_grid(g, kernels->P, V, scratch, kStaticScratchBytes, &w);
    return grid_dispatch(g, kernels, uvw, reinterpret_cast<const float2*>(vis), weight, V, w,
                         reinterpret_cast<float2*>(grid), stats, st);
}
