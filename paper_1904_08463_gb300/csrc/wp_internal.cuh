// Internal declarations of the GB300 w-projection library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/wproj.h"

namespace wp {

// NVTX range around each C-ABI call (free unless a profiler is attached), so that tools can
// attribute kernels to the library call that launched them.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#define WP_RANGE(name) ::wp::NvtxRange wp_nvtx_range_(name)

// ---------------------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------------------
void set_last_error(const char* where, const char* what);
int cuda_fail(const char* where, cudaError_t e);

#define WP_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::wp::cuda_fail(#call, e_);       \
    } while (0)

#define WP_LAUNCH_CHECK(name)                                           \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return ::wp::cuda_fail(name, e_);        \
    } while (0)

// ---------------------------------------------------------------------------------------
// checked build (-DWP_CHECK_BOUNDS)
// ---------------------------------------------------------------------------------------
// The kernels test the index of each main buffer access against the buffer's extent with
// in_bounds(); in the checked build an access outside is skipped and the first one of each
// translation unit recorded in a device word of that unit (site << 48 | low 48 bits of the
// index); wp_bounds_status gathers the words of every unit.  In the default build in_bounds is
// a constant true and every check compiles away.
enum BoundSite : int {
    BS_CACHE_WRITE = 1,   // resample: a staged row copied into the kernel cache
    BS_TAP = 2,           // a gridder or degridder reading a tap of its plane's cache block
    BS_GRID = 3,          // a grid cell read or written
    BS_VIS = 4,           // a visibility written by a degridder
};
int bounds_register(int (*read)(unsigned long long* first, bool clear));
#ifdef WP_CHECK_BOUNDS
namespace {
__device__ unsigned long long g_bounds_first;       // one per translation unit
int bounds_read_unit(unsigned long long* first, bool clear) {
    WP_CUDA(cudaMemcpyFromSymbol(first, g_bounds_first, sizeof(unsigned long long)));
    if (clear) {
        const unsigned long long zero = 0;
        WP_CUDA(cudaMemcpyToSymbol(g_bounds_first, &zero, sizeof(zero)));
    }
    return WP_OK;
}
const int g_bounds_registered = bounds_register(&bounds_read_unit);
}  // namespace
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int site) {
    if ((uint64_t)i < (uint64_t)n) return true;
    atomicCAS(&g_bounds_first, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(int64_t, int64_t, int) { return true; }
#endif

// ---------------------------------------------------------------------------------------
// derived geometry of a plan
// ---------------------------------------------------------------------------------------
struct Geom {
    int N, os, s_max, s_min, R, r_pad, k_out, interp, kernelgen, fft_m, grid_tile, grid_method;
    double dl, du, r_max, tau;
};

int make_geom(const wp_plan* plan, Geom* g);
int check_grid_args(const wp_plan* plan, const wp_wkernels* k, const float* uvw, int64_t V, void* workspace,
                    size_t workspace_bytes, Geom* g, bool gridding = false, bool with_workspace = true);
int check_device_public();   // WP_OK when the current device is sm_103

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Padded plane count: the matrix product works on 2*P_pad columns, a multiple of 128.
inline int p_pad(int P) { return (int)round_up(P, 64); }

// ---------------------------------------------------------------------------------------
// workspace carving: consecutive 256-byte aligned segments
// ---------------------------------------------------------------------------------------
struct Carver {
    char* base;
    size_t off;
    size_t cap;
    explicit Carver(void* b, size_t c) : base((char*)b), off(0), cap(c) {}
    template <class T>
    T* take(size_t count) {
        off = (size_t)round_up((int64_t)off, 256);
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    bool fits() const { return off <= cap; }
};

// Kernel-generation workspace segments.
struct KgWork {
    float* h32;        // [k_out][r_pad] FP32 transform matrix
    float* h_hi;       // [k_out][r_pad] TF32 high part
    float* h_lo;       // [k_out][r_pad] TF32 low part
    uint16_t* hb_hi;   // [k_out][r_pad] BF16 high part (BF16x3 route)
    uint16_t* hb_lo;   // [k_out][r_pad] BF16 low part
    uint16_t* hb_lo2;  // [k_out][r_pad] BF16 third part (BF16x6 route)
    float* band;       // [65][k_out] spline inverse band (row d holds A^-1[k][k + d - 32])
    double* nm1;       // [R] n - 1 = sqrt(1 - r_i^2) - 1 at the radial nodes
    float2* nm1f;      // [R] the same as an unevaluated float pair (hi, lo)
    float2* ps_nm1;    // [M * M] n - 1 at the workspace pixels as float pairs (projection route)
    float2* ps_x;      // [P][M os] projected, zero-padded lines, transformed in place (projection route)
    float* f32;        // [2 P_pad][r_pad] image-domain functions (FP32 path)
    float* f_hi;       // [2 P_pad][r_pad]
    float* f_lo;       // [2 P_pad][r_pad]
    uint16_t* fb_hi;   // [2 P_pad][r_pad] BF16 split of the image-domain functions (BF16x3 route)
    uint16_t* fb_lo;   // [2 P_pad][r_pad]
    uint16_t* fb_lo2;  // [2 P_pad][r_pad] third part (BF16x6 route)
    float* gct;        // [2 P_pad][k_out] radial-line gradient rows (re, im) for the adjoint
    int*   status;     // [4]
};
size_t carve_kg(const Geom& g, int P, void* ws, size_t bytes, KgWork* out);

// Gridding workspace segments.
struct GridWork {
    int T, ntx, ntiles;
    int64_t nbins;
    int*    count;      // [nbins + 1]   per (plane, centre tile) counts, then exclusive scan
    int*    cursor;     // [nbins]
    int*    key;        // [V]           bin key, -1 when dropped
    int4*   rec;        // [V]           unsorted records
    int4*   srec;       // [V]           records sorted by bin
    float2* svis;       // [V]           weighted visibilities sorted by bin
    int*    flags;      // [nbins + 1]   work-item flags, then exclusive scan
    int*    items;      // [nbins]       compacted work items (plane * ntiles + tile)
    int*    scan_tmp;   // scan scratch
    int*    ctrl;       // [8]  [0] item cursor, [1] item count, [2] status
    double* red;        // [2]  weight sum, drops (per call)
    int*    seff;       // [P]  effective supports of the call (clamped, fitted to the cache layout)
    // slot gridder (grid_method 9) only; zero-sized otherwise
    uint64_t* skey;     // [V]  (plane, Morton cell) keys, and their ping-pong copy
    uint64_t* skey_alt;
    uint32_t* sidx;     // [V]  visibility index carried by the sort, and its copy
    uint32_t* sidx_alt;
    int*    rs_hist;    // radix-sort digit histograms
    int*    rs_tmp;     // their scan scratch
    int*    vstart;     // [P + 1] first sorted visibility of each plane
    int*    icount;     // [P + 1] work items per plane, then
    int*    istart;     // [P + 1] their exclusive scan
};
size_t carve_grid(const Geom& g, int P, int64_t V, void* ws, size_t bytes, GridWork* out);

// ---------------------------------------------------------------------------------------
// launchers (return WP_OK or an error code; all asynchronous on `st`)
// ---------------------------------------------------------------------------------------
// The kernel tap at fine offset (dx, dy) (units du/os) from the plane's radial line staged in
// shared memory as {y.re, y.im, m.re, m.im} per sample, slot k at skew(k) (XOR swizzle within
// each group of 8: neighbouring taps are up to os samples apart on the line).  The radius test
// q = dx^2 + dy^2 <= lim2 = (os S)^2 is exact on integers; x = sqrt(q) only picks the spline
// interval and its weights, which are continuous across interval ends.  Shared by the
// resample (cache) and the on-the-fly gridder, so both produce the same bits.
// ---------------------------------------------------------------------------------------
#ifdef __CUDACC__
// The support a kernel may use for plane p of a cache laid out by `offsets`: S itself when
// its os^2 (2S+1)^2 taps fit the plane's block [offsets[p], offsets[p+1]) -- always, for a
// layout from wp_kernel_layout of the same supports -- else the largest support that fits, or
// 0 (skip the plane) when not even S = 1 does.  Every path that turns (support, offsets) into
// cache indices goes through it -- the resample and the 2D-FFT extraction per block, gridding
// and degridding through the per-call effective supports that binning computes -- so a
// caller's inconsistent layout gives wrong taps for that plane but no access outside its
// block.
__device__ __forceinline__ int fit_support(int S, int os, const int64_t* __restrict__ offsets, int p) {
    const int64_t blk = offsets[p + 1] - offsets[p];
    const int64_t os2 = (int64_t)os * os;
    int s = S;
    while (s >= 1 && os2 * (2 * (int64_t)s + 1) * (2 * (int64_t)s + 1) > blk) --s;
    return s;
}

__device__ __forceinline__ int skew(int k) { return k ^ ((k >> 3) & 7); }

// Binning decisions of one visibility (Alg. 1 / Alg. 2: nearest |w| plane, ties to the lower
// index; conjugation for w < 0, Section 4.1; grid cell and oversampling offset), all in FP64
// with explicitly rounded operations so that every binning kernel takes the same decisions:
//   t = rint((u/du + N/2) os), iu = floor(t/os), fu = t - iu os   (same for v).
// wps: the P ascending plane values (shared memory); support: the call's effective supports
// (0 when a plane's cache block holds none).  Returns false (dropped) when u, v or w is not
// finite, the plane is unusable, or any tap of the (2S+1)^2 footprint leaves [0, N)^2.
__device__ __forceinline__ bool bin_decide(const float* __restrict__ uvw, int64_t k, int P, const double* wps,
                                           const int32_t* __restrict__ support, int N, double du, int os,
                                           int* p_out, int* iu_out, int* iv_out, int* fu_out, int* fv_out,
                                           int* conj_out) {
    const double u = (double)uvw[3 * k], v = (double)uvw[3 * k + 1], w = (double)uvw[3 * k + 2];
    const double aw = fabs(w);
    // lower_bound over the ascending plane values, then nearest of the two neighbours
    int lo = 0, hi = P;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (wps[mid] < aw) lo = mid + 1; else hi = mid;
    }
    int p;
    if (lo == 0) p = 0;
    else if (lo == P) p = P - 1;
    else {
        const double dl_ = fabs(aw - wps[lo - 1]);
        const double dh_ = fabs(aw - wps[lo]);
        p = (dh_ < dl_) ? lo : lo - 1;          // ties -> lower index
    }
    const double uc = __dadd_rn(__ddiv_rn(u, du), (double)(N / 2));
    const double vc = __dadd_rn(__ddiv_rn(v, du), (double)(N / 2));
    const double tu = rint(__dmul_rn(uc, (double)os));
    const double tv = rint(__dmul_rn(vc, (double)os));
    const double giu = floor(__ddiv_rn(tu, (double)os));
    const double giv = floor(__ddiv_rn(tv, (double)os));
    const int S = support[p];
    const bool ok = S >= 1 && isfinite(u) && isfinite(v) && isfinite(w) && (giu - S >= 0.0) &&
                    (giu + S <= (double)(N - 1)) && (giv - S >= 0.0) && (giv + S <= (double)(N - 1));
    *p_out = p;
    *conj_out = (w < 0.0) ? 1 : 0;
    if (ok) {
        *iu_out = (int)giu;
        *iv_out = (int)giv;
        *fu_out = (int)(tu - giu * (double)os);
        *fv_out = (int)(tv - giv * (double)os);
    } else {
        *iu_out = *iv_out = *fu_out = *fv_out = 0;
    }
    return ok;
}

// Spline interval of radius sqrt(q) on the unit-spaced line: k = round(x - 1/2) through the
// float mantissa (1.5 * 2^23) from an approximate x = q rsqrt(q) -- an off-by-one next to an
// integer radius is harmless, the interpolant being continuous there.  The offset keeps the
// part of the root that FP32 x drops, by one Newton step: sqrt(q) = x + e / (2x) + O(e^2/x^3)
// with the residual e = q - x^2 = (q - k^2) - (x - k)(x + k), where q - k^2 is exact in
// integers (q itself may exceed 2^24) and x - k is exact (Sterbenz), so e carries ~1e-3 at
// most of absolute error and a = (x - k) + e r / 2 keeps ~1e-7 absolute accuracy at radii of
// thousands of samples, where x - k alone keeps ~3e-5.  No division.
__device__ __forceinline__ void tap_interval(int q, int& k, float& a) {
    const float qf = (float)q;
    const float r = rsqrtf(fmaxf(qf, 1.0f));
    const float x = qf * r;                          // q = 0 gives 0
    const float tt = (x - 0.5f) + 12582912.0f;
    k = __float_as_int(tt) - 0x4B400000;
    const float kf = tt - 12582912.0f;               // k as a float, exactly
    const float xk = x - kf;
    const float e = fmaf(-xk, x + kf, (float)(q - k * k));
    a = fmaf(e, 0.5f * r, xk);
}

template <bool CUBIC>
__device__ __forceinline__ float2 resample_tap(const float4* __restrict__ line, int dx, int dy, int lim2) {
    const int q = dx * dx + dy * dy;
    float2 out = make_float2(0.0f, 0.0f);
    if (q <= lim2) {
        int k;
        float a;
        tap_interval(q, k, a);
        const float b = 1.0f - a;
        const float4 L0 = line[skew(k)];
        const float4 L1 = line[skew(k + 1)];
        out.x = fmaf(b, L0.x, a * L1.x);
        out.y = fmaf(b, L0.y, a * L1.y);
        if (CUBIC) {
            const float cb = (b * b - 1.0f) * b * (1.0f / 6.0f);
            const float ca = (a * a - 1.0f) * a * (1.0f / 6.0f);
            out.x = fmaf(cb, L0.z, fmaf(ca, L1.z, out.x));
            out.y = fmaf(cb, L0.w, fmaf(ca, L1.w, out.y));
        }
    }
    return out;
}
#endif

// ---------------------------------------------------------------------------------------
int kg_prepare(const Geom& g, const KgWork& w, cudaStream_t st);
int kg_screen(const Geom& g, const KgWork& w, const float* taper, const double* w_planes, int P,
              cudaStream_t st);
int kg_gemm_fp32(const Geom& g, const KgWork& w, int P, float2* radial, cudaStream_t st);
int kg_gemm_tf32x3(const Geom& g, const KgWork& w, int P, float2* radial, int* status,
                   cudaStream_t st);
int kg_gemm_bf16x3(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st);
int kg_gemm_bf16x6(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st);
int kg_gemm_tf32x3_ex(const Geom& g, const KgWork& w, int P, float2* radial, int* status, cudaStream_t st,
                      long long budget, int withhold_loads);
int kg_ps_prepare(const Geom& g, const KgWork& w, cudaStream_t st);
int kg_projslice(const Geom& g, const KgWork& w, const float* taper, const double* w_planes, int P,
                 float2* radial, cudaStream_t st);
int kg_trunc_spline(const Geom& g, const KgWork& w, int P, const float2* radial, float2* spline_m,
                    int32_t* support, cudaStream_t st);
int kg_resample(const Geom& g, int P, const float2* radial, const float2* spline_m,
                const int32_t* support, const int64_t* offsets, float2* cache, cudaStream_t st);

int exclusive_scan_i32(const int* in, int* out, int64_t n, int* tmp, cudaStream_t st);
size_t scan_tmp_ints(int64_t n);

// stable LSD radix sort (sort.cu); KT = uint32_t or uint64_t, vals may be NULL
int64_t radix_sort_tiles(int64_t n);
size_t radix_sort_hist_ints(int64_t n);
template <class KT>
int radix_sort(KT* keys, uint32_t* vals, KT* keys_alt, uint32_t* vals_alt, int64_t n, int bits, int* hist,
               int* scan_tmp, cudaStream_t st, bool* in_alt);

int grid_bin(const Geom& g, const wp_wkernels* k, const float* uvw, const float2* vis,
             const float* weight, int64_t V, const GridWork& w, cudaStream_t st);
int grid_bin_noscatter(const Geom& g, const wp_wkernels* kern, const float* uvw, const float* weight, int64_t V,
                       const GridWork& w, cudaStream_t st);
int item_flags(const Geom& g, const wp_wkernels* kern, const GridWork& w, cudaStream_t st);
// persistent multi-job gridding (grid_batch.cu)
size_t grid_batch_ctrl_bytes();
long long grid_batch_budget();
int grid_batch_prepare(const Geom& g, const wp_wkernels* kern, const float* uvw, const float* weight, int64_t V,
                       const GridWork& w, cudaStream_t st);
int grid_batch_run(int n_jobs, const Geom* geoms, const wp_wkernels* kerns, const float* const* vis,
                   const float* const* weight, const int64_t* Vs, const GridWork* works, float* const* grids,
                   const uint32_t* const* sidx, int tile, void* bws, long long budget, int withhold, int fused,
                   cudaStream_t st);
int grid_run(const Geom& g, const wp_wkernels* k, const GridWork& w, float2* grid, double* stats,
             cudaStream_t st);
int write_items(int64_t n, const GridWork& w, cudaStream_t st);   // compact live items (flags scanned into cursor)
void k_fit_supports_launch(const Geom& g, const wp_wkernels* kern, const GridWork& w, cudaStream_t st);
int add_stats(double* stats, const double* red, cudaStream_t st);
size_t slot_hist_ints(int64_t V);
int grid_slot(const Geom& g, const wp_wkernels* kern, const float* uvw, const float2* vis, const float* weight,
              int64_t V, const GridWork& w, float2* grid, double* stats, cudaStream_t st);
int grid_slot_prepare(const Geom& g, const wp_wkernels* kern, const float* uvw, const float* weight, int64_t V,
                      const GridWork& w, cudaStream_t st, const uint32_t** idx_sorted, bool degrid = false);
// one gridding call on a carved workspace, by plan.grid_method (wp_grid and wp_grid_static)
int grid_dispatch(const Geom& g, const wp_wkernels* kern, const float* uvw, const float2* vis, const float* weight,
                  int64_t V, const GridWork& w, float2* grid, double* stats, cudaStream_t st);
int degrid_slot(const Geom& g, const wp_wkernels* kern, const float* uvw, int64_t V, const GridWork& w,
                const float2* grid, float2* vis_out, cudaStream_t st);
int grid_run_group(const Geom& g, const wp_wkernels* k, const GridWork& w, float2* grid, cudaStream_t st);
int degrid_run(const Geom& g, const wp_wkernels* k, int64_t V, const GridWork& w, const float2* grid,
               float2* vis_out, cudaStream_t st);

int image_dirty(const Geom& g, const float* taper, float2* grid, double wsum, const double* wsum_dev,
                float* image, cudaStream_t st);
int image_to_grid(const Geom& g, const float* taper, const float* image, double wsum, float2* grid,
                  cudaStream_t st);
void release_fft_plans();

size_t fft_workspace_bytes(const Geom& g, int P);
int fft_wkernels(const Geom& g, const float* taper, const double* w_planes, int P, const int32_t* support,
                 const int64_t* offsets, int circular, void* ws, size_t ws_bytes, float2* cache,
                 cudaStream_t st);
void release_fft_kernelgen_plans();
void release_ps_plans();

// plane values (planes.cu)
size_t plane_values_workspace_bytes(int64_t V);
int plane_values(const float* uvw, int64_t V, int P, void* ws, size_t bytes, double* out, cudaStream_t st);

// differentiation (grad.cu)
struct GradWork {
    int*    count2;     // [P os^2 + 1] visibilities per (plane, sub-kernel), then exclusive scan
    int*    cursor2;    // [P os^2 + 1]
    int*    uv2;        // [V] cell (iu | iv << 16) of each regrouped visibility
    float4* g4;         // [V] (g, s g), s = -1 for w < 0
    int*    scan_tmp;
};
size_t carve_grad(const Geom& g, int P, int64_t V, void* ws, size_t bytes, GradWork* out);
int grad_radial_run(const Geom& g, const wp_wkernels* kern, const GridWork& w, const GradWork& gw,
                    const float2* gvis, const float2* grid, float2* gC, float2* gM, cudaStream_t st);
int hankel_adjoint_run(const Geom& g, const KgWork& w, int P, const double* w_planes, const float2* gC,
                       const float2* gM, float* grad_taper, cudaStream_t st);
int launch_image_adjoint(const Geom& g, const float* taper, const float* image, const float2* F, double wsum,
                         float* grad_image, float* grad_taper, cudaStream_t st);
int image_adjoint(const Geom& g, const float* taper, const float* image, float2* grid_g, double wsum,
                  float* grad_image, float* grad_taper, cudaStream_t st);

}  // namespace wp
