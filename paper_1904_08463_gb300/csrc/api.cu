// C ABI entry points of libwproj.so: argument validation on the host, workspace carving,
// and the launch sequence of each call.  Nothing here computes on the host beyond sizes.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "wp_internal.cuh"

#define WP_VERSION 100   // 0.1.0

namespace wp {

static thread_local char g_err[512] = "";

void set_last_error(const char* where, const char* what) {
    snprintf(g_err, sizeof(g_err), "%s: %s", where, what);
}

int cuda_fail(const char* where, cudaError_t e) {
    set_last_error(where, cudaGetErrorString(e));
    return WP_ERR_CUDA;
}

int make_geom(const wp_plan* plan, Geom* g) {
    if (!plan || !g) return WP_ERR_NULL;
    const int N = plan->image_size;
    if (N < 16 || N > 65536 || (N & 1)) return WP_ERR_PLAN;
    if (!(plan->cell_size > 0.0) || !(0.5 * N * plan->cell_size < 1.0)) return WP_ERR_PLAN;
    if (plan->oversampling < 1 || plan->oversampling > 16) return WP_ERR_PLAN;
    if (plan->max_support < 1 || plan->max_support > 511) return WP_ERR_PLAN;
    if (2 * plan->max_support + 1 > N) return WP_ERR_PLAN;
    if (plan->min_support < 1 || plan->min_support > plan->max_support) return WP_ERR_PLAN;
    if (!(plan->trunc_frac < 1.0)) return WP_ERR_PLAN;
    if (plan->radial_samples < 8 || plan->radial_samples > 65536) return WP_ERR_PLAN;
    if (plan->interp != WP_INTERP_CUBIC && plan->interp != WP_INTERP_LINEAR) return WP_ERR_PLAN;
    if (plan->kernelgen != WP_KG_FP32 && plan->kernelgen != WP_KG_TF32X3 && plan->kernelgen != WP_KG_BF16X3 &&
        plan->kernelgen != WP_KG_BF16X6 && plan->kernelgen != WP_KG_PROJSLICE)
        return WP_ERR_PLAN;
    if (plan->grid_tile != 0 && plan->grid_tile != 32 && plan->grid_tile != 64) return WP_ERR_PLAN;
    if (plan->grid_method < 0 || plan->grid_method > 9) return WP_ERR_PLAN;
    g->N = N;
    g->dl = plan->cell_size;
    g->du = 1.0 / ((double)N * plan->cell_size);
    g->r_max = 0.5 * (double)N * plan->cell_size;
    g->os = plan->oversampling;
    g->s_max = plan->max_support;
    g->s_min = plan->min_support;
    g->tau = plan->trunc_frac;
    g->R = plan->radial_samples;
    g->r_pad = (int)round_up(plan->radial_samples, 64);   // whole K slices for TF32 (32) and BF16 (64)
    g->k_out = (int)round_up((int64_t)plan->oversampling * (plan->max_support + 2), 128);
    g->interp = plan->interp;
    g->kernelgen = plan->kernelgen;
    g->grid_tile = plan->grid_tile ? plan->grid_tile : 64;
    g->grid_method = plan->grid_method;
    int m = 1;
    while (m < 2 * plan->max_support + 1) m *= 2;
    g->fft_m = m;
    return WP_OK;
}

size_t carve_kg(const Geom& g, int P, void* ws, size_t bytes, KgWork* out) {
    Carver c(ws, bytes);
    const size_t hk = (size_t)g.k_out * g.r_pad;
    const size_t fk = (size_t)2 * p_pad(P) * g.r_pad;
    KgWork w;
    w.h32 = c.take<float>(hk);
    w.h_hi = c.take<float>(hk);
    w.h_lo = c.take<float>(hk);
    // every route's buffers, so that one prepared workspace serves all kernelgen routes
    w.hb_hi = c.take<uint16_t>(hk);
    w.hb_lo = c.take<uint16_t>(hk);
    w.hb_lo2 = c.take<uint16_t>(hk);
    w.band = c.take<float>((size_t)g.k_out * 65);
    w.nm1 = c.take<double>((size_t)g.r_pad);
    w.nm1f = c.take<float2>((size_t)g.r_pad);
    w.ps_nm1 = c.take<float2>((size_t)g.fft_m * g.fft_m);
    w.ps_x = c.take<float2>((size_t)P * g.fft_m * g.os);
    w.f32 = c.take<float>(fk);
    w.f_hi = c.take<float>(fk);
    w.f_lo = c.take<float>(fk);
    w.fb_hi = c.take<uint16_t>(fk);
    w.fb_lo = c.take<uint16_t>(fk);
    w.fb_lo2 = c.take<uint16_t>(fk);
    w.gct = c.take<float>((size_t)2 * p_pad(P) * g.k_out);
    w.status = c.take<int>(64);
    if (out) *out = w;
    return (size_t)round_up((int64_t)c.off, 256);
}

size_t carve_grid(const Geom& g, int P, int64_t V, void* ws, size_t bytes, GridWork* out) {
    Carver c(ws, bytes);
    GridWork w;
    w.T = (g.grid_method == 2) ? 32 : g.grid_tile;    // the warp-private gridder uses 32 x 32 tiles
    w.ntx = (g.N + w.T - 1) / w.T;
    w.ntiles = w.ntx * w.ntx;
    w.nbins = (int64_t)P * w.ntiles;
    w.count = c.take<int>((size_t)w.nbins + 1);
    w.cursor = c.take<int>((size_t)w.nbins + 1);
    w.key = c.take<int>((size_t)V);
    w.rec = c.take<int4>((size_t)V);
    w.srec = c.take<int4>((size_t)V);
    w.svis = c.take<float2>((size_t)V);
    w.flags = c.take<int>((size_t)w.nbins + 1);
    w.items = c.take<int>((size_t)w.nbins + 1);
    w.scan_tmp = c.take<int>(scan_tmp_ints(w.nbins + 1));
    w.ctrl = c.take<int>(64);
    w.red = c.take<double>(8);
    w.seff = c.take<int>((size_t)P);
    const bool slot = (g.grid_method == 9);
    const size_t vs = slot ? (size_t)V : 0, ps = slot ? (size_t)P + 1 : 0;
    const size_t hist = slot ? radix_sort_hist_ints(V) : 0;
    w.skey = c.take<uint64_t>(vs);
    w.skey_alt = c.take<uint64_t>(vs);
    w.sidx = c.take<uint32_t>(vs);
    w.sidx_alt = c.take<uint32_t>(vs);
    w.rs_hist = c.take<int>(hist);
    w.rs_tmp = c.take<int>(slot ? scan_tmp_ints((int64_t)hist) : 0);
    w.vstart = c.take<int>(ps);
    w.icount = c.take<int>(ps);
    w.istart = c.take<int>(ps);
    if (out) *out = w;
    return (size_t)round_up((int64_t)c.off, 256);
}

static int check_device() {
    static int cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WP_ERR_CUDA;
    if (dev < 0 || dev >= 64) return WP_ERR_DEVICE;
    if (cached[dev] == 0) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return WP_ERR_CUDA;
        cached[dev] = (major == 10 && minor == 3) ? 1 : -1;
    }
    return cached[dev] == 1 ? WP_OK : WP_ERR_DEVICE;
}

static bool aligned256(const void* p) { return ((uintptr_t)p & 255u) == 0; }

int check_device_public() { return check_device(); }

// the bounds records of the checked build, one reader per translation unit
static std::vector<int (*)(unsigned long long*, bool)>& bounds_units() {
    static std::vector<int (*)(unsigned long long*, bool)> units;
    return units;
}

int bounds_register(int (*read)(unsigned long long* first, bool clear)) {
    bounds_units().push_back(read);
    return 0;
}

}  // namespace wp

using namespace wp;

extern "C" {

int wp_version(void) { return WP_VERSION; }

const char* wp_last_error_string(void) { return g_err; }

const char* wp_strerror(int code) {
    switch (code) {
        case WP_OK: return "ok";
        case WP_ERR_NULL: return "a required pointer is NULL";
        case WP_ERR_SIZE: return "a size or count argument is out of range";
        case WP_ERR_PLAN: return "inconsistent plan";
        case WP_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
        case WP_ERR_CUDA: return "CUDA or cuFFT call failed";
        case WP_ERR_TIMEOUT: return "a bounded device-side wait expired";
        case WP_ERR_DEVICE: return "current device is not sm_103 (GB300)";
        case WP_ERR_UNSUPPORTED: return "request not supported by the library";
        case WP_ERR_INFLIGHT: return "a bounded wait expired with device work still in flight (context suspect)";
        default: return "unknown status";
    }
}

int wp_bounds_status(uint64_t* first, int32_t clear) {
#ifdef WP_CHECK_BOUNDS
    if (!first) return WP_ERR_NULL;
    *first = 0;
    WP_CUDA(cudaDeviceSynchronize());
    for (auto read : bounds_units()) {
        unsigned long long v = 0;
        int rc = read(&v, clear != 0);
        if (rc) return rc;
        if (*first == 0 && v != 0) *first = v;
    }
    return WP_OK;
#else
    (void)first;
    (void)clear;
    return WP_ERR_UNSUPPORTED;
#endif
}

void wp_release(void) {
    release_fft_plans();
    release_fft_kernelgen_plans();
    release_ps_plans();
}

int wp_plan_geometry(const wp_plan* plan, wp_geometry* geom) {
    if (!plan || !geom) return WP_ERR_NULL;
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    geom->k_out = g.k_out;
    geom->r_pad = g.r_pad;
    geom->fft_workspace = g.fft_m;
    geom->reserved = 0;
    geom->du = g.du;
    geom->r_max = g.r_max;
    return WP_OK;
}

int wp_kernel_layout(const wp_plan* plan, int32_t P, const int32_t* support_host, int64_t* offsets_host) {
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (!support_host || !offsets_host) return WP_ERR_NULL;
    if (P < 1) return WP_ERR_SIZE;
    const int64_t os2 = (int64_t)g.os * g.os;
    offsets_host[0] = 0;
    for (int p = 0; p < P; ++p) {
        int s = support_host[p];
        if (s < 1 || s > g.s_max) return WP_ERR_SIZE;
        offsets_host[p + 1] = offsets_host[p] + os2 * (2 * s + 1) * (2 * s + 1);
    }
    return WP_OK;
}

int wp_kernel_layout_max(const wp_plan* plan, int32_t P, int64_t* offsets_host) {
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (!offsets_host) return WP_ERR_NULL;
    if (P < 1) return WP_ERR_SIZE;
    const int64_t blk = (int64_t)g.os * g.os * (2 * g.s_max + 1) * (2 * g.s_max + 1);
    for (int p = 0; p <= P; ++p) offsets_host[p] = blk * p;
    return WP_OK;
}

size_t wp_kernelgen_workspace_bytes(const wp_plan* plan, int32_t P) {
    Geom g;
    if (make_geom(plan, &g) || P < 1) return 0;
    return carve_kg(g, P, nullptr, 0, nullptr);
}

int wp_kernelgen_prepare(const wp_plan* plan, int32_t P, void* workspace, size_t workspace_bytes,
                         void* stream) {
    WP_RANGE("wp_kernelgen_prepare");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!workspace) return WP_ERR_NULL;
    if (!aligned256(workspace) || workspace_bytes < carve_kg(g, P, nullptr, 0, nullptr)) return WP_ERR_WORKSPACE;
    if ((rc = check_device())) return rc;
    KgWork w;
    carve_kg(g, P, workspace, workspace_bytes, &w);
    return kg_prepare(g, w, (cudaStream_t)stream);
}

int wp_hankel_radial(const wp_plan* plan, const float* taper, const double* w_planes, int32_t P,
                     void* workspace, size_t workspace_bytes, float* radial, float* spline_m,
                     int32_t* support, void* stream) {
    WP_RANGE("wp_hankel_radial");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!taper || !w_planes || !workspace || !radial) return WP_ERR_NULL;
    if (g.interp == WP_INTERP_CUBIC && !spline_m) return WP_ERR_NULL;
    if (g.tau > 0.0 && !support) return WP_ERR_NULL;
    if (!aligned256(workspace) || workspace_bytes < carve_kg(g, P, nullptr, 0, nullptr)) return WP_ERR_WORKSPACE;
    if ((rc = check_device())) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    KgWork w;
    carve_kg(g, P, workspace, workspace_bytes, &w);
    if (g.kernelgen == WP_KG_PROJSLICE) {
        rc = kg_projslice(g, w, taper, w_planes, P, reinterpret_cast<float2*>(radial), st);
    } else {
        if ((rc = kg_screen(g, w, taper, w_planes, P, st))) return rc;
        if (g.kernelgen == WP_KG_TF32X3)
            rc = kg_gemm_tf32x3(g, w, P, reinterpret_cast<float2*>(radial), w.status, st);
        else if (g.kernelgen == WP_KG_BF16X3)
            rc = kg_gemm_bf16x3(g, w, P, reinterpret_cast<float2*>(radial), w.status, st);
        else if (g.kernelgen == WP_KG_BF16X6)
            rc = kg_gemm_bf16x6(g, w, P, reinterpret_cast<float2*>(radial), w.status, st);
        else
            rc = kg_gemm_fp32(g, w, P, reinterpret_cast<float2*>(radial), st);
    }
    if (rc) return rc;
    return kg_trunc_spline(g, w, P, reinterpret_cast<const float2*>(radial),
                           reinterpret_cast<float2*>(spline_m), support, st);
}

int wp_kernelgen_status(const wp_plan* plan, int32_t P, void* workspace, size_t workspace_bytes,
                        int32_t* status_host, void* stream) {
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!workspace || !status_host) return WP_ERR_NULL;
    if (!aligned256(workspace) || workspace_bytes < carve_kg(g, P, nullptr, 0, nullptr)) return WP_ERR_WORKSPACE;
    KgWork w;
    carve_kg(g, P, workspace, workspace_bytes, &w);
    WP_CUDA(cudaMemcpyAsync(status_host, w.status, sizeof(int32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    WP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return WP_OK;
}

int wp_selftest_bounded_wait(const wp_plan* plan, int32_t P, void* workspace, size_t workspace_bytes,
                             float* radial, int32_t* status_host, void* stream) {
    WP_RANGE("wp_selftest_bounded_wait");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!workspace || !radial || !status_host) return WP_ERR_NULL;
    if (!aligned256(workspace) || workspace_bytes < carve_kg(g, P, nullptr, 0, nullptr)) return WP_ERR_WORKSPACE;
    if ((rc = check_device())) return rc;
    KgWork w;
    carve_kg(g, P, workspace, workspace_bytes, &w);
    // loads withheld, 2e7-cycle (~10 ms) budget: the first wait of every CTA expires
    rc = kg_gemm_tf32x3_ex(g, w, P, reinterpret_cast<float2*>(radial), w.status, (cudaStream_t)stream,
                           20000000LL, 1);
    if (rc) return rc;
    WP_CUDA(cudaMemcpyAsync(status_host, w.status, sizeof(int32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    WP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return WP_OK;
}

int wp_resample(const wp_plan* plan, const float* radial, const float* spline_m, int32_t P,
                const int32_t* support, const int64_t* offsets, float* cache, void* stream) {
    WP_RANGE("wp_resample");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!radial || !support || !offsets || !cache) return WP_ERR_NULL;
    if (g.interp == WP_INTERP_CUBIC && !spline_m) return WP_ERR_NULL;
    if ((uintptr_t)cache & 7u) return WP_ERR_SIZE;    // complex64 taps
    if ((rc = check_device())) return rc;
    return kg_resample(g, P, reinterpret_cast<const float2*>(radial),
                       reinterpret_cast<const float2*>(spline_m), support, offsets,
                       reinterpret_cast<float2*>(cache), (cudaStream_t)stream);
}

int wp_make_wkernels(const wp_plan* plan, const float* taper, const double* w_planes, int32_t P,
                     int32_t* support, const int64_t* offsets, void* workspace, size_t workspace_bytes,
                     float* radial, float* spline_m, float* cache, void* stream) {
    WP_RANGE("wp_make_wkernels");
    if (!support || !offsets || !cache) return WP_ERR_NULL;
    int rc = wp_hankel_radial(plan, taper, w_planes, P, workspace, workspace_bytes, radial, spline_m,
                              support, stream);
    if (rc) return rc;
    return wp_resample(plan, radial, spline_m, P, support, offsets, cache, stream);
}

int wp_make_wkernels_owned(const wp_plan* plan, const float* taper, const double* w_planes, int32_t P,
                           const int32_t* support, wp_wkernels* out, void* stream) {
    WP_RANGE("wp_make_wkernels_owned");
    if (!out) return WP_ERR_NULL;
    memset(out, 0, sizeof(*out));
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!taper || !w_planes) return WP_ERR_NULL;
    const bool trunc = g.tau > 0.0;
    if (!trunc && !support) return WP_ERR_NULL;
    for (int p = 0; p < P; ++p) {
        if (!(w_planes[p] >= 0.0) || (p > 0 && w_planes[p] < w_planes[p - 1])) return WP_ERR_SIZE;
        if (!trunc && (support[p] < 1 || support[p] > g.s_max)) return WP_ERR_SIZE;
    }
    if ((rc = check_device())) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const bool cubic = (g.interp == WP_INTERP_CUBIC);
    // every allocation is released on any error path
    std::vector<void*> held;
    auto alloc = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) return cuda_fail("cudaMalloc", e);
        held.push_back(*p);
        return WP_OK;
    };
    auto fail = [&](int code) {
        cudaStreamSynchronize(st);
        for (void* p : held) cudaFree(p);
        memset(out, 0, sizeof(*out));
        return code;
    };
    const size_t ws_bytes = carve_kg(g, P, nullptr, 0, nullptr);
    void *ws = nullptr, *d_w = nullptr, *d_sup = nullptr, *d_off = nullptr, *d_rad = nullptr, *d_spl = nullptr,
         *d_cache = nullptr;
    const size_t line_bytes = (size_t)P * g.k_out * sizeof(float2);
    if ((rc = alloc(&ws, ws_bytes)) || (rc = alloc(&d_w, (size_t)P * sizeof(double))) ||
        (rc = alloc(&d_sup, (size_t)P * sizeof(int32_t))) || (rc = alloc(&d_off, (size_t)(P + 1) * sizeof(int64_t))) ||
        (rc = alloc(&d_rad, line_bytes)) || (cubic && (rc = alloc(&d_spl, line_bytes))))
        return fail(rc);
    cudaError_t e = cudaMemcpyAsync(d_w, w_planes, (size_t)P * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !trunc)
        e = cudaMemcpyAsync(d_sup, support, (size_t)P * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(cuda_fail("cudaMemcpyAsync", e));
    if ((rc = wp_kernelgen_prepare(plan, P, ws, ws_bytes, stream))) return fail(rc);
    if ((rc = wp_hankel_radial(plan, taper, (const double*)d_w, P, ws, ws_bytes, (float*)d_rad, (float*)d_spl,
                               trunc ? (int32_t*)d_sup : nullptr, stream)))
        return fail(rc);
    std::vector<int32_t> sup_h((size_t)P);
    std::vector<int64_t> off_h((size_t)P + 1);
    if (trunc) {
        e = cudaMemcpyAsync(sup_h.data(), d_sup, (size_t)P * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(cuda_fail("support read-back", e));
    } else {
        memcpy(sup_h.data(), support, (size_t)P * sizeof(int32_t));
    }
    if ((rc = wp_kernel_layout(plan, P, sup_h.data(), off_h.data()))) return fail(rc);
    if ((rc = alloc(&d_cache, (size_t)off_h[P] * sizeof(float2)))) return fail(rc);
    e = cudaMemcpyAsync(d_off, off_h.data(), (size_t)(P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(cuda_fail("cudaMemcpyAsync", e));
    if ((rc = wp_resample(plan, (const float*)d_rad, (const float*)d_spl, P, (const int32_t*)d_sup,
                          (const int64_t*)d_off, (float*)d_cache, stream)))
        return fail(rc);
    e = cudaStreamSynchronize(st);   // host vectors above must outlive their copies
    if (e != cudaSuccess) return fail(cuda_fail("cudaStreamSynchronize", e));
    cudaFree(ws);
    out->P = P;
    out->flags = WP_KERNELS_OWNED;
    out->w_planes = (const double*)d_w;
    out->support = (const int32_t*)d_sup;
    out->offsets = (const int64_t*)d_off;
    out->cache = (const float*)d_cache;
    out->radial = (const float*)d_rad;
    out->spline_m = (const float*)d_spl;
    return WP_OK;
}

int wp_free_kernels(wp_wkernels* k) {
    if (!k) return WP_ERR_NULL;
    if (!(k->flags & WP_KERNELS_OWNED)) {
        set_last_error("wp_free_kernels", "kernel set not allocated by wp_make_wkernels_owned");
        return WP_ERR_UNSUPPORTED;
    }
    WP_CUDA(cudaDeviceSynchronize());
    const void* ptrs[6] = {k->w_planes, k->support, k->offsets, k->cache, k->radial, k->spline_m};
    for (const void* p : ptrs)
        if (p) WP_CUDA(cudaFree(const_cast<void*>(p)));
    memset(k, 0, sizeof(*k));
    return WP_OK;
}

size_t wp_fft_workspace_bytes(const wp_plan* plan, int32_t P) {
    Geom g;
    if (make_geom(plan, &g) || P < 1) return 0;
    return fft_workspace_bytes(g, P);
}

int wp_fft_wkernels(const wp_plan* plan, const float* taper, const double* w_planes, int32_t P,
                    const int32_t* support, const int64_t* offsets, int32_t circular, void* workspace,
                    size_t workspace_bytes, float* cache, void* stream) {
    WP_RANGE("wp_fft_wkernels");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!taper || !w_planes || !support || !offsets || !workspace || !cache) return WP_ERR_NULL;
    if (!aligned256(workspace) || workspace_bytes < fft_workspace_bytes(g, P)) return WP_ERR_WORKSPACE;
    if ((int64_t)g.fft_m * g.os > 32768) return WP_ERR_SIZE;
    if ((rc = check_device())) return rc;
    return fft_wkernels(g, taper, w_planes, P, support, offsets, circular, workspace, workspace_bytes,
                        reinterpret_cast<float2*>(cache), (cudaStream_t)stream);
}

size_t wp_plane_values_workspace_bytes(int64_t V) {
    if (V < 1 || V > 2147483647LL) return 0;
    return plane_values_workspace_bytes(V);
}

int wp_plane_values(const float* uvw, int64_t V, int32_t P, void* workspace, size_t workspace_bytes,
                    double* w_planes, void* stream) {
    WP_RANGE("wp_plane_values");
    if (!uvw || !workspace || !w_planes) return WP_ERR_NULL;
    if (V < 1 || V > 2147483647LL || P < 1 || P > V) return WP_ERR_SIZE;
    if (!aligned256(workspace) || workspace_bytes < plane_values_workspace_bytes(V)) return WP_ERR_WORKSPACE;
    int rc = check_device();
    if (rc) return rc;
    return plane_values(uvw, V, P, workspace, workspace_bytes, w_planes, (cudaStream_t)stream);
}

size_t wp_grid_workspace_bytes(const wp_plan* plan, int32_t P, int64_t V) {
    Geom g;
    if (make_geom(plan, &g) || P < 1 || V < 0) return 0;
    return carve_grid(g, P, V, nullptr, 0, nullptr);
}

}  // extern "C"

// One gridding call on a carved workspace: the slot gridder (9) bins along a Morton curve of
// each plane; every other method bins by (plane, tile) and runs from its item list.
int wp::grid_dispatch(const Geom& g, const wp_wkernels* kern, const float* uvw, const float2* vis,
                      const float* weight, int64_t V, const GridWork& w, float2* grid, double* stats,
                      cudaStream_t st) {
    if (g.grid_method == 9) return grid_slot(g, kern, uvw, vis, weight, V, w, grid, stats, st);
    int rc = grid_bin(g, kern, uvw, vis, weight, V, w, st);
    if (rc) return rc;
    return grid_run(g, kern, w, grid, stats, st);
}

// Argument checks of every call that bins visibilities.  with_workspace = false skips the
// caller-workspace checks (the allocation-free gridder supplies its own scratch).
int wp::check_grid_args(const wp_plan* plan, const wp_wkernels* k, const float* uvw, int64_t V,
                        void* workspace, size_t workspace_bytes, Geom* g, bool gridding, bool with_workspace) {
    int rc = make_geom(plan, g);
    if (rc) return rc;
    if (!k || (with_workspace && !workspace)) return WP_ERR_NULL;
    if (k->P < 1 || k->P > 8192) return WP_ERR_SIZE;
    if (!k->w_planes || !k->support || !k->offsets) return WP_ERR_NULL;
    if (gridding && g->grid_method == 4) {      // taps from the radial lines, no cache
        if (!k->radial || (g->interp == WP_INTERP_CUBIC && !k->spline_m)) return WP_ERR_NULL;
    } else if (!k->cache) {
        return WP_ERR_NULL;
    }
    if (V < 0 || V > 2147483647LL) return WP_ERR_SIZE;
    if (V > 0 && !uvw) return WP_ERR_NULL;
    if ((int64_t)k->P * ((g->N + 63) / 64) * ((g->N + 63) / 64) >= 2147483647LL) return WP_ERR_SIZE;
    if (with_workspace &&
        (!aligned256(workspace) || workspace_bytes < carve_grid(*g, k->P, V, nullptr, 0, nullptr)))
        return WP_ERR_WORKSPACE;
    return check_device();
}

extern "C" {

int wp_grid(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw, const float* vis,
            const float* weight, int64_t V, void* workspace, size_t workspace_bytes, float* grid,
            double* stats, void* stream) {
    WP_RANGE("wp_grid");
    Geom g;
    int rc = check_grid_args(plan, kernels, uvw, V, workspace, workspace_bytes, &g, true);
    if (rc) return rc;
    if (!grid || (V > 0 && !vis)) return WP_ERR_NULL;
    cudaStream_t st = (cudaStream_t)stream;
    GridWork w;
    carve_grid(g, kernels->P, V, workspace, workspace_bytes, &w);
    return grid_dispatch(g, kernels, uvw, reinterpret_cast<const float2*>(vis), weight, V, w,
                         reinterpret_cast<float2*>(grid), stats, st);
}

int wp_degrid(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw, const float* grid,
              int64_t V, void* workspace, size_t workspace_bytes, float* vis_out, void* stream) {
    WP_RANGE("wp_degrid");
    Geom g;
    int rc = check_grid_args(plan, kernels, uvw, V, workspace, workspace_bytes, &g);
    if (rc) return rc;
    if (!grid || (V > 0 && !vis_out)) return WP_ERR_NULL;
    cudaStream_t st = (cudaStream_t)stream;
    GridWork w;
    carve_grid(g, kernels->P, V, workspace, workspace_bytes, &w);
    if (g.grid_method == 9)      // slot degridder: the adjoint walk over Morton-sorted planes
        return degrid_slot(g, kernels, uvw, V, w, reinterpret_cast<const float2*>(grid),
                           reinterpret_cast<float2*>(vis_out), st);
    if ((rc = grid_bin(g, kernels, uvw, nullptr, nullptr, V, w, st))) return rc;
    return degrid_run(g, kernels, V, w, reinterpret_cast<const float2*>(grid),
                      reinterpret_cast<float2*>(vis_out), st);
}

size_t wp_grad_workspace_bytes(const wp_plan* plan, int32_t P, int64_t V) {
    Geom g;
    if (make_geom(plan, &g) || P < 1 || V < 0) return 0;
    return carve_grid(g, P, V, nullptr, 0, nullptr) + carve_grad(g, P, V, nullptr, 0, nullptr);
}

int wp_grad_radial(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw, const float* grad_vis,
                   const float* grid, int64_t V, void* workspace, size_t workspace_bytes, float* grad_radial,
                   float* grad_spline_m, void* stream) {
    WP_RANGE("wp_grad_radial");
    Geom g;
    int rc = check_grid_args(plan, kernels, uvw, V, workspace, workspace_bytes, &g);
    if (rc) return rc;
    if (!grid || !grad_radial || (V > 0 && !grad_vis)) return WP_ERR_NULL;
    if (g.interp == WP_INTERP_CUBIC && !grad_spline_m) return WP_ERR_NULL;
    if (workspace_bytes < wp_grad_workspace_bytes(plan, kernels->P, V)) return WP_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    GridWork w;
    const size_t gb = carve_grid(g, kernels->P, V, workspace, workspace_bytes, &w);
    GradWork gw;
    carve_grad(g, kernels->P, V, static_cast<char*>(workspace) + gb, workspace_bytes - gb, &gw);
    if ((rc = grid_bin(g, kernels, uvw, nullptr, nullptr, V, w, st))) return rc;
    return grad_radial_run(g, kernels, w, gw, reinterpret_cast<const float2*>(grad_vis),
                           reinterpret_cast<const float2*>(grid), reinterpret_cast<float2*>(grad_radial),
                           reinterpret_cast<float2*>(grad_spline_m), st);
}

int wp_hankel_adjoint(const wp_plan* plan, const double* w_planes, int32_t P, void* workspace,
                      size_t workspace_bytes, const float* grad_radial, const float* grad_spline_m,
                      float* grad_taper, void* stream) {
    WP_RANGE("wp_hankel_adjoint");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (P < 1 || P > 65536) return WP_ERR_SIZE;
    if (!w_planes || !workspace || !grad_radial || !grad_taper) return WP_ERR_NULL;
    if (g.interp == WP_INTERP_CUBIC && !grad_spline_m) return WP_ERR_NULL;
    if (g.kernelgen == WP_KG_PROJSLICE) return WP_ERR_UNSUPPORTED;   // the adjoint is the matrix route's
    if (!aligned256(workspace) || workspace_bytes < carve_kg(g, P, nullptr, 0, nullptr)) return WP_ERR_WORKSPACE;
    if ((rc = check_device())) return rc;
    KgWork w;
    carve_kg(g, P, workspace, workspace_bytes, &w);
    return hankel_adjoint_run(g, w, P, w_planes, reinterpret_cast<const float2*>(grad_radial),
                              reinterpret_cast<const float2*>(grad_spline_m), grad_taper, (cudaStream_t)stream);
}

int wp_image_adjoint(const wp_plan* plan, const float* taper, const float* image, float* grid_g,
                     double weight_sum, float* grad_image, float* grad_taper, void* stream) {
    WP_RANGE("wp_image_adjoint");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (!taper || !image || !grid_g || !grad_image || !grad_taper) return WP_ERR_NULL;
    if (!(weight_sum > 0.0)) return WP_ERR_SIZE;
    if ((rc = check_device())) return rc;
    return image_adjoint(g, taper, image, reinterpret_cast<float2*>(grid_g), weight_sum, grad_image, grad_taper,
                         (cudaStream_t)stream);
}

int wp_dirty_image(const wp_plan* plan, const float* taper, float* grid, double weight_sum, float* image,
                   void* stream) {
    WP_RANGE("wp_dirty_image");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (!taper || !grid || !image) return WP_ERR_NULL;
    if (!(weight_sum > 0.0)) return WP_ERR_SIZE;
    if ((rc = check_device())) return rc;
    return image_dirty(g, taper, reinterpret_cast<float2*>(grid), weight_sum, nullptr, image, (cudaStream_t)stream);
}

int wp_dirty_image_stats(const wp_plan* plan, const float* taper, float* grid, const double* weight_sum_dev,
                         float* image, void* stream) {
    WP_RANGE("wp_dirty_image_stats");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (!taper || !grid || !weight_sum_dev || !image) return WP_ERR_NULL;
    if ((uintptr_t)weight_sum_dev & 7u) return WP_ERR_SIZE;
    if ((rc = check_device())) return rc;
    return image_dirty(g, taper, reinterpret_cast<float2*>(grid), 0.0, weight_sum_dev, image, (cudaStream_t)stream);
}

int wp_image_to_grid(const wp_plan* plan, const float* taper, const float* image, double weight_sum,
                     float* grid, void* stream) {
    WP_RANGE("wp_image_to_grid");
    Geom g;
    int rc = make_geom(plan, &g);
    if (rc) return rc;
    if (!taper || !grid || !image) return WP_ERR_NULL;
    if (!(weight_sum > 0.0)) return WP_ERR_SIZE;
    if ((rc = check_device())) return rc;
    return image_to_grid(g, taper, image, weight_sum, reinterpret_cast<float2*>(grid), (cudaStream_t)stream);
}

}  // extern "C"
