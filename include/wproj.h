/*
 * wproj.h -- C ABI of the GB300 w-projection library (libwproj.so).
 *
 * Hankel-accelerated w-projection (Lucas, Skipper & Scaife, "Fast W-Projection for
 * Wide-field Imaging", MNRAS 2019): per-|w|-plane oversampled convolution kernels are
 * generated by an order-0 Hankel transform of the radially symmetric product
 * (anti-aliasing taper) x (w-screen) instead of a 2D FFT (Section 4.3, Alg. 2), then
 * visibilities are convolved onto the uv-grid with the kernel of their nearest plane
 * (Alg. 1 / Alg. 2 gridding step) and inverse transformed to a dirty image (Section 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument is a DEVICE pointer unless its comment says "host".
 *    Device memory is owned by the caller; the library allocates no device memory
 *    except cuFFT plans/work areas (wp_dirty_image, wp_image_to_grid, wp_fft_wkernels, the
 *    projection route of wp_hankel_radial), which it caches per device, size and stream
 *    until wp_release() -- one per stream, so that calls overlapping on different streams
 *    never share a work area; the first such call on a stream creates its plan and must
 *    therefore come before any stream capture that uses that stream -- and the fixed
 *    scratch array of wp_grid_static.
 *  - Complex values are interleaved float pairs (re, im) -- the layout of CUDA's
 *    float2 / cuFloatComplex / torch.complex64.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*; NULL is
 *    the legacy default stream) and returns 0 (WP_OK) when all launches were queued.
 *    Invalid arguments are detected on the host BEFORE any launch and return a negative
 *    WP_ERR_* code with nothing launched.  WP_ERR_CUDA reports a failed launch (the
 *    CUDA error string is available from wp_last_error_string()).  Device-side data
 *    errors (e.g. a bounded wait that expired) are reported through the `status` word
 *    of the calls that take one.
 *  - Units: cell_size in radians (direction-cosine units), u, v, w in wavelengths.
 *
 * Geometry (Sections 3-5 of the paper):
 *    N = image_size, dl = cell_size, FOV = N dl, du = 1/FOV (uv cell),
 *    r_max = FOV/2 (radius of the circular image region), os = oversampling,
 *    S = kernel support (half-width in cells; full width 2S+1),
 *    R = radial_samples, radial nodes r_i = (i + 1/2) r_max / R,
 *    K_out = os (S_max + 2) rounded up to a multiple of 128 radial kernel samples at
 *            rho_k = k du / os.
 */
#ifndef WPROJ_H
#define WPROJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define WP_OK              0
#define WP_ERR_NULL       -1   /* a required pointer is NULL                          */
#define WP_ERR_SIZE       -2   /* a size/count argument is out of range               */
#define WP_ERR_PLAN       -3   /* inconsistent wp_plan fields                         */
#define WP_ERR_WORKSPACE  -4   /* workspace too small or misaligned                   */
#define WP_ERR_CUDA       -5   /* a CUDA / cuFFT call failed                          */
#define WP_ERR_TIMEOUT    -6   /* a bounded device-side wait expired                  */
#define WP_ERR_DEVICE     -7   /* current device is not sm_103 (GB300)                */
#define WP_ERR_UNSUPPORTED -8  /* valid request outside what the library implements     */
#define WP_ERR_INFLIGHT   -9   /* a bounded wait expired and the kernel had to exit with a
                                  copy or tensor-core operation still in flight (a drain
                                  wait ran out as well): results are void and the CUDA
                                  context should be treated as suspect (reset it)         */

/* plan.interp (Section 4.3.2: linear or cubic-spline interpolation of the radial line) */
#define WP_INTERP_CUBIC    0
#define WP_INTERP_LINEAR   1

/* plan.kernelgen: how the radial line is obtained */
#define WP_KG_FP32         0   /* Hankel transform as FP32 SIMT matrix product          */
#define WP_KG_TF32X3       1   /* Hankel transform on tcgen05 tensor cores, TF32 hi/lo
                                  split (3 products), FP32 accumulation in TMEM          */
#define WP_KG_BF16X3       3   /* Hankel transform on tcgen05 tensor cores, BF16 hi/lo
                                  split (3 products, kind::f16 at twice the TF32 rate),
                                  FP32 accumulation in TMEM: operand split error ~2e-6
                                  relative (TF32x3: ~3e-8)                               */
#define WP_KG_BF16X6       4   /* Hankel transform on tcgen05 tensor cores, each operand
                                  split into three BF16 parts (all 24 bits of FP32), the
                                  six products of order <= 2 (kind::f16): TF32x3's
                                  accuracy at the same tensor time                      */
#define WP_KG_PROJSLICE    2   /* Hankel transform by the projection-slice theorem
                                  (Section 4.3.1, Alg. 2 steps 4-12): the taper x screen
                                  on the undersampled M x M workspace (Section 4.2) summed
                                  over one axis, zero-padded by os, 1D FFT; the radial
                                  line is the v = 0 slice of the 2D-FFT route's transform */

/*
 * Imager settings (Section 5: image size, cell size, oversampling, maximum support,
 * truncation percentage, interpolation type; Section 4.2: workspace undersampling).
 * All fields are host values.
 */
typedef struct wp_plan {
    int32_t image_size;     /* N, even, 16 <= N <= 65536                               */
    double  cell_size;      /* dl (radians), N*dl/2 < 1                                */
    int32_t oversampling;   /* os, 1 <= os <= 16                                       */
    int32_t max_support;    /* S_max, 1 <= S_max <= 511 (Section 5: 127 <-> 255x255)    */
    int32_t min_support;    /* S_min, 1 <= S_min <= S_max                              */
    double  trunc_frac;     /* tau in (0, 1): support = last radius with |C| >= tau*max
                               (Section 3.1, default 0.01); <= 0: supports are given   */
    int32_t radial_samples; /* R, 8 <= R <= 65536                                      */
    int32_t interp;         /* WP_INTERP_CUBIC | WP_INTERP_LINEAR                      */
    int32_t kernelgen;      /* WP_KG_FP32 | WP_KG_TF32X3 | WP_KG_BF16X3 | WP_KG_BF16X6 |
                               WP_KG_PROJSLICE                                           */
    int32_t grid_tile;      /* gridding tile side in cells: 0 (default, 64), 32 or 64    */
    int32_t grid_method;    /* 0 (default): register tile, lanes own grid cells;
                               1: shared-memory tile, footprint spread over the lanes;
                               2: per-warp shared-memory 32 x 32 tiles, groups of 8 planes
                               per work item (grid_tile ignored);
                               3: shared-memory tile, each warp owning every 8th row, lanes
                               across the footprint's columns (no atomics in the tile);
                               4: as 3, each tap interpolated on the fly from the plane's
                               radial line (wp_wkernels.radial / spline_m) instead of
                               read from the cache;
                               5: as 3 over groups of 8 consecutive planes per work item
                               (one flush of the tile for the whole group);
                               6: groups of 8 planes, each warp's rows of the tile held in
                               registers, lanes across the columns;
                               7, 8: as 3, with 2 (7) or 4 (8) consecutive visibilities of a
                               bin applied per shared-memory read-modify-write;
                               9: slots -- each lane owns footprint positions modulo 2S+1 and
                               sums its taps in registers over visibilities sorted along a
                               Morton curve of their cells, writing to the grid only when
                               its cell changes (grid_tile ignored).
                               grid_tile and grid_method are tuning choices only: the
                               results agree to FP32 rounding order                      */
} wp_plan;

/* Derived sizes of a plan (host struct filled by wp_plan_geometry). */
typedef struct wp_geometry {
    int32_t k_out;          /* radial kernel samples K_out (multiple of 128)           */
    int32_t r_pad;          /* R rounded up to a multiple of 32                        */
    int32_t fft_workspace;  /* M of the 2D-FFT route: power of two >= 2 S_max + 1      */
    int32_t reserved;
    double  du;             /* uv cell, wavelengths                                   */
    double  r_max;          /* radius of the circular image region                    */
} wp_geometry;

/*
 * A generated kernel set (all DEVICE pointers, caller-owned; the struct itself is a
 * host value).  Plane p's cache block starts at complex element offsets[p] of `cache`
 * and holds os*os sub-kernels [fv][fu], each (2 S_p + 1)^2 taps [jy][jx], where the
 * tap (jx, jy) of sub-kernel (fu, fv) is the kernel at uv offset
 * (jx - S_p - fu/os, jy - S_p - fv/os) cells.  Kernels are for +|w|; a visibility with
 * w < 0 uses the complex conjugate (Section 4.1).  offsets must give every block room for
 * its support (wp_kernel_layout of the same supports, or wp_kernel_layout_max); a plane whose
 * block is smaller is read and written with the largest support the block holds, or skipped
 * when not even S = 1 fits, so a mismatched layout yields wrong taps for that plane but no
 * access outside its block.
 */
#define WP_KERNELS_OWNED (1 << 30)   /* wp_wkernels.flags: arrays allocated by
                                        wp_make_wkernels_owned (free with wp_free_kernels) */
typedef struct wp_wkernels {
    int32_t        P;         /* number of |w| planes                                  */
    int32_t        flags;     /* 0 for caller-owned arrays; WP_KERNELS_OWNED           */
    const double*  w_planes;  /* [P] plane |w| values, ascending, >= 0                 */
    const int32_t* support;   /* [P] support S_p, min_support <= S_p <= max_support    */
    const int64_t* offsets;   /* [P+1] complex-element offsets into cache              */
    const float*   cache;     /* interleaved complex taps                              */
    const float*   radial;    /* [P][K_out] complex radial lines (wp_hankel_radial);
                                 read only by gridding with grid_method 4, which then
                                 needs no cache (cache may be NULL)                     */
    const float*   spline_m;  /* [P][K_out] spline second derivatives (cubic, method 4) */
} wp_wkernels;

/* ---- plan helpers (host only, no device work) -------------------------------------- */

/* Validate `plan` and fill `geom`.  Returns WP_OK or WP_ERR_NULL / WP_ERR_PLAN. */
int wp_plan_geometry(const wp_plan* plan, wp_geometry* geom);

/*
 * Compact cache layout for known supports: offsets[p+1] = offsets[p] + os^2 (2 S_p + 1)^2
 * (host arrays: support [P] in, offsets [P+1] out).  With truncation on (trunc_frac > 0)
 * the supports are only known after wp_hankel_radial; a caller that does not want to
 * read them back sizes every block for max_support (wp_kernel_layout_max).
 */
int wp_kernel_layout(const wp_plan* plan, int32_t P, const int32_t* support_host,
                     int64_t* offsets_host);
int wp_kernel_layout_max(const wp_plan* plan, int32_t P, int64_t* offsets_host);

/* ---- kernel generation (Alg. 2 with the Hankel transform, Section 4.3) ------------- */

/* Bytes of scratch that wp_hankel_radial / wp_make_wkernels need for P planes. */
size_t wp_kernelgen_workspace_bytes(const wp_plan* plan, int32_t P);

/*
 * Once per plan geometry (Section 4.3: the transform matrix does not depend on the plane, so it is built once):
 * builds in `workspace` the K_out x R transform matrix H[k][i] = du^2 2 pi r_i dr
 * J0(2 pi rho_k r_i) (J0 evaluated in FP64 on the device, stored as FP32, as a TF32 hi/lo
 * pair and as a BF16 hi/lo pair), the table of n - 1 at the M x M workspace pixels of the
 * projection route (FP64, stored as float pairs) and the band of the inverse of the spline
 * system -- the tables of every kernelgen route, so one prepared workspace serves them all
 * (the workspace layout does not depend on plan->kernelgen).  Must precede
 * wp_hankel_radial / wp_make_wkernels on that workspace; they then accept any P' whose
 * workspace size still fits.  Synchronizes `stream` (a small host table is uploaded).
 */
int wp_kernelgen_prepare(const wp_plan* plan, int32_t P, void* workspace,
                         size_t workspace_bytes, void* stream);

/*
 * Radial kernel lines of P planes: for each plane p (|w| = w_planes[p]):
 *   f_p(r_i) = taper[i] * exp(+2 pi j w_p (sqrt(1 - r_i^2) - 1))          (Eq. 9, adjoint sign)
 *   radial[p][k] = du^2 * sum_i 2 pi r_i dr J0(2 pi rho_k r_i) f_p(r_i)  (Eq. 12, matrix form)
 * computed as one batched matrix product (K_out x R) x (R x 2P).  With kernelgen ==
 * WP_KG_PROJSLICE the line is instead the v = 0 slice of the 2D transform of the same
 * function sampled on the undersampled M x M workspace (Section 4.2), obtained by the
 * projection-slice theorem (Section 4.3.1): column sums, zero padding to M os, 1D FFT,
 * scaled by (FOV/M)^2 du^2; sample k is taken at index k mod (M os).  Also writes the cubic
 * spline second derivatives of each line (Section 4.3.2; clamped slope 0 at rho = 0,
 * natural at rho_{K_out-1}) and, if plan->trunc_frac > 0, the support of each plane
 * (Section 3.1: last rho_k with |radial| >= trunc_frac * max, ceil to whole cells,
 * clamped to [S_min, S_max]).
 *   taper     [R] float, t(r_i) (the radial anti-aliasing function)
 *   w_planes  [P] double, >= 0
 *   workspace scratch of wp_kernelgen_workspace_bytes(plan, P) bytes, 256-byte aligned,
 *             prepared by wp_kernelgen_prepare with the same plan geometry
 *   radial    [P][K_out] complex out;  spline_m [P][K_out] complex out (may be NULL when
 *             plan->interp == WP_INTERP_LINEAR);  support [P] int32 out (ignored, may be
 *             NULL, when trunc_frac <= 0)
 */
int wp_hankel_radial(const wp_plan* plan, const float* taper, const double* w_planes,
                     int32_t P, void* workspace, size_t workspace_bytes, float* radial,
                     float* spline_m, int32_t* support, void* stream);

/*
 * Device-side status of the last kernel-generation call on `workspace` (synchronizes
 * `stream`): 0, or WP_ERR_TIMEOUT when a bounded wait of the tensor-core transform expired
 * (its output is then left unwritten, and the CUDA context stays usable), or WP_ERR_INFLIGHT
 * when, after such an expiry, the kernel could not see its own copies land within a second
 * budget either and exited with them in flight (context suspect).
 */
int wp_kernelgen_status(const wp_plan* plan, int32_t P, void* workspace, size_t workspace_bytes,
                        int32_t* status_host, void* stream);

/*
 * Self-test of that failure path: runs the tensor-core transform with its tile loads
 * withheld and a ~10 ms wait budget, so every CTA's first wait expires; writes the
 * resulting device status to *status_host (expected WP_ERR_TIMEOUT) and synchronizes.
 * Nothing faults or hangs; `radial` ([P][K_out] complex) is not written.
 */
int wp_selftest_bounded_wait(const wp_plan* plan, int32_t P, void* workspace,
                             size_t workspace_bytes, float* radial, int32_t* status_host,
                             void* stream);

/*
 * Oversampled kernel cache from the radial lines (Section 4.3.2 and the cache step of
 * Alg. 2): tap (jx, jy) of sub-kernel (fu, fv) of plane p is the interpolated radial
 * line at radius x = sqrt((os (jx - S) - fu)^2 + (os (jy - S) - fv)^2) samples, and 0 when
 * x > os S (the truncated line rotated about rho = 0 has circular support).
 *   radial, spline_m  as written by wp_hankel_radial (spline_m unused for linear)
 *   support [P] int32 (values outside [1, S_max] are clamped), offsets [P+1] int64 (device),
 *   cache out (device memory), 8-byte aligned (WP_ERR_SIZE otherwise).  A plane whose block
 *   [offsets[p], offsets[p+1]) is too small for its support gets the largest support that
 *   fits (or is left unwritten): nothing is written outside the blocks.
 */
int wp_resample(const wp_plan* plan, const float* radial, const float* spline_m, int32_t P,
                const int32_t* support, const int64_t* offsets, float* cache, void* stream);

/*
 * wp_hankel_radial followed by wp_resample, for supports fixed by the caller
 * (plan->trunc_frac <= 0; support [P] is then an input) or computed by truncation
 * (support is then an output and offsets must give every block room for max_support).
 */
int wp_make_wkernels(const wp_plan* plan, const float* taper, const double* w_planes,
                     int32_t P, int32_t* support, const int64_t* offsets, void* workspace,
                     size_t workspace_bytes, float* radial, float* spline_m, float* cache,
                     void* stream);

/*
 * The same kernels in device memory the library allocates: a complete kernel set from the
 * problem statement alone (image geometry, taper, w-planes, oversampling, support).  The
 * call allocates with cudaMalloc -- it is neither allocation-free nor capturable -- and
 * synchronizes `stream` before returning.
 *   taper     device [R] float
 *   w_planes  HOST [P] plane |w| values, ascending, >= 0 (copied to the device)
 *   support   HOST [P] supports in [1, max_support] when plan->trunc_frac <= 0; NULL when
 *             the truncation rule (Section 3.1) picks them on the device -- they are then
 *             read back to lay the cache out compactly
 *   out       filled with device pointers to w_planes, support, offsets, cache, radial and
 *             spline_m (NULL for linear interpolation), all owned by the library, and flags
 *             = WP_KERNELS_OWNED; usable by every gridding call; release with wp_free_kernels
 * On an error nothing stays allocated and *out is zeroed.
 */
int wp_make_wkernels_owned(const wp_plan* plan, const float* taper, const double* w_planes,
                           int32_t P, const int32_t* support, wp_wkernels* out, void* stream);

/*
 * Frees a kernel set made by wp_make_wkernels_owned and zeroes *kernels.  Synchronizes the
 * device first, so that no queued kernel still reads it.  A set whose flags lack
 * WP_KERNELS_OWNED (caller-owned arrays) is refused with WP_ERR_UNSUPPORTED and left as is.
 */
int wp_free_kernels(wp_wkernels* kernels);

/* ---- standard kernel generation by 2D FFT (the comparator; Alg. 1, Section 4.2) ------ */

/* Bytes of scratch for wp_fft_wkernels: a batch of zero-padded (M os)^2 complex workspaces
   (as many planes as fit in 1 GiB, at least one) and an M^2 table. */
size_t wp_fft_workspace_bytes(const wp_plan* plan, int32_t P);

/*
 * Kernel cache by the standard route: per plane the image-domain product taper x w-screen
 * t(r) exp(+2 pi j w (sqrt(1 - r^2) - 1)) is sampled on the M x M workspace spanning the
 * field of view (M = power of two >= 2 S_max + 1, Section 4.2; t linearly interpolated
 * between the radial nodes, 0 outside r_max), zero padded to (M os)^2 (Alg. 1, oversampling
 * by padding), transformed (cuFFT C2C forward, batched), scaled by (FOV/M)^2 du^2, and tap
 * (jx, jy) of sub-kernel (fu, fv) is read at fine offset (os (jx - S) - fu, os (jy - S) - fv).
 * With circular != 0 taps beyond radius S are zeroed (the Hankel route's support shape).
 * Same cache layout as wp_resample; supports are inputs (no truncation in this route).
 *   taper [R] float, w_planes [P] double, support [P] int32, offsets [P+1] int64 (device);
 *   workspace wp_fft_workspace_bytes(plan, P) bytes, 256-byte aligned; cache out.
 * Uses cached batched cuFFT plans (freed by wp_release).
 */
int wp_fft_wkernels(const wp_plan* plan, const float* taper, const double* w_planes, int32_t P,
                    const int32_t* support, const int64_t* offsets, int32_t circular,
                    void* workspace, size_t workspace_bytes, float* cache, void* stream);

/* ---- w-plane values (Alg. 1 / Alg. 2 steps 1-3) ------------------------------------- */

/* Bytes of scratch for wp_plane_values with V visibilities. */
size_t wp_plane_values_workspace_bytes(int64_t V);

/*
 * Plane values as the paper's default: sort |w| of all V visibilities, cut the sorted list
 * into P equal-count chunks (the first V mod P chunks hold one more) and take each chunk's
 * mean (FP64 sums of the float32 |w|).  Result ascending, ready for wp_wkernels.w_planes.
 *   uvw [V][3] float; w_planes [P] double out; 1 <= P <= V.
 */
int wp_plane_values(const float* uvw, int64_t V, int32_t P, void* workspace,
                    size_t workspace_bytes, double* w_planes, void* stream);

/* ---- gridding (Alg. 1 / Alg. 2 gridding step) and its adjoint ----------------------- */

/* Bytes of scratch that wp_grid / wp_degrid need for V visibilities. */
size_t wp_grid_workspace_bytes(const wp_plan* plan, int32_t P, int64_t V);

/*
 * Convolutional gridding: for every visibility k (u, v, w = uvw[k][0..2]):
 *   plane p = nearest |w| plane (ties -> lower index), conj = (w < 0),
 *   t = rint((u/du + N/2) os), iu = floor(t/os), fu = t - iu os   (same for v),
 *   grid[iv - S + jy][iu - S + jx] += weight[k] vis[k] K            for jx, jy in [0, 2S],
 * K = tap (jx, jy) of sub-kernel (fu, fv) of plane p, conjugated when w < 0.  These
 * integer decisions are taken in FP64.  A visibility whose footprint leaves [0, N)^2 is
 * dropped.  The grid (rows v, columns u) is ACCUMULATED into (not cleared).
 *   uvw [V][3] float, vis [V] complex, weight [V] float or NULL (all 1)
 *   workspace  wp_grid_workspace_bytes(plan, P, V) bytes, 256-byte aligned
 *   grid       [N][N] complex in/out
 *   stats      double[2] or NULL: stats[0] += sum of weights gridded,
 *              stats[1] += number of dropped visibilities
 */
int wp_grid(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw,
            const float* vis, const float* weight, int64_t V, void* workspace,
            size_t workspace_bytes, float* grid, double* stats, void* stream);

/*
 * Degridding, the adjoint of wp_grid with unit weights:
 *   vis_out[k] = sum_taps conj(K) grid[iv - S + jy][iu - S + jx]   (0 if dropped)
 * Same binning rules and workspace as wp_grid.  plan.grid_method 9 walks the slots (each holds
 * the grid value of its cell and reloads it only when the cell changes); any other value uses a
 * warp per visibility.  The results agree to FP32 summation order.
 */
int wp_degrid(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw,
              const float* grid, int64_t V, void* workspace, size_t workspace_bytes,
              float* vis_out, void* stream);

/*
 * Allocation-free gridding.  This entry point has no counterpart in the paper; it exists
 * for callers that cannot allocate device memory -- for example an imaging pipeline that
 * reserves all of HBM for its own pools at start-up and forbids later allocations, or a
 * host framework whose plug-ins may only use memory they are handed -- and therefore
 * cannot provide the scratch that wp_grid takes.
 *  - Same arguments and result as wp_grid, minus the workspace: the scratch is one array of
 *    WP_GRID_STATIC_SCRATCH_BYTES (64 MiB) compiled into the library.
 *  - A problem whose scratch need (wp_grid_workspace_bytes) exceeds that size is rejected
 *    with WP_ERR_SIZE before any launch (roughly 1.5 million visibilities fit with a
 *    256^2 grid and 16 planes; fewer with large grids and many planes).
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current.  CUDA loads the module holding the array lazily, so it is this
 *    first call that commits the 64 MiB on that device (held until the process exits), not
 *    the loading of the library: a caller that reserves its memory pools up front must make
 *    the first call before reserving them -- a call with V = 0 (uvw and vis may be NULL)
 *    does the set-up and grids nothing -- and before any stream capture.
 *  - No cudaMalloc, cudaFree or allocating library routine is called.
 *  - All calls share the one array and it keeps the previous call's contents; each call
 *    clears what must start at zero.  Calls that overlap on the GPU (other streams or host
 *    threads) race on the array: the caller must serialise them.
 */
#define WP_GRID_STATIC_SCRATCH_BYTES (64ull << 20)
int wp_grid_static(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw,
                   const float* vis, const float* weight, int64_t V, float* grid,
                   double* stats, void* stream);

/* ---- many independent problems in one persistent launch ----------------------------- */

/*
 * One gridding job of a batch: the arguments of one wp_grid call, by value.  The batch grids a
 * job with the slot method when plan.grid_method is 9, otherwise with the row-owned shared-tile
 * method (grid_method 3) whatever plan.grid_method says; plan.grid_tile (0 = 64, or 32) must be
 * the same for every row-owned job of a batch.
 *   workspace  wp_grid_workspace_bytes(plan with grid_method 9 or 3, P, V) bytes, 256-byte
 *              aligned (the job's own; jobs never share one)
 */
#define WP_GRID_BATCH_MAX_JOBS 128
typedef struct wp_grid_job {
    wp_plan        plan;
    wp_wkernels    kernels;
    const float*   uvw;
    const float*   vis;
    const float*   weight;
    int64_t        V;
    void*          workspace;
    size_t         workspace_bytes;
    float*         grid;
    double*        stats;
} wp_grid_job;

/* Bytes of the batch's own control workspace (queue, per-job counters, status). */
size_t wp_grid_batch_workspace_bytes(void);

/*
 * Grids n_jobs independent problems (1 <= n_jobs <= WP_GRID_BATCH_MAX_JOBS; jobs: host array)
 * with the same result per job as wp_grid.  Each job is binned as in wp_grid up to its list of
 * live work items; then persistent launches pull work from one device queue per gridder kind
 * (row-owned, slot) -- every job's ordering of its records first (the scatter into bin order,
 * or for slot jobs the gather into the sorted order), then every job's gridding items (a block
 * per row-owned (plane, tile) item, a warp per slot item), in the order of `jobs` (put large jobs
 * first) -- so small problems fill the GPU beside large ones with no per-job tail.  The
 * orderings and the items run as two launches per kind.  Argument errors of any job are
 * reported before anything is launched.  Calls overlapping on the GPU must use different batch
 * workspaces and job workspaces.
 */
int wp_grid_batch(int32_t n_jobs, const wp_grid_job* jobs, void* batch_workspace,
                  size_t batch_workspace_bytes, void* stream);

/*
 * The same gridding as wp_grid_batch with the orderings and the items of each kind in ONE
 * launch, each job's ordering chunks queued right before its items: an item waits for its job's
 * orderings, done by blocks that took them from the queue earlier.  The wait is bounded (about a
 * second of SM clock); on expiry the item is skipped and the batch status records
 * WP_ERR_TIMEOUT (read it with wp_grid_batch_status).  Measured about 4 % slower than
 * wp_grid_batch on 48 problems (its items read their records through L2).
 */
int wp_grid_batch_fused(int32_t n_jobs, const wp_grid_job* jobs, void* batch_workspace,
                        size_t batch_workspace_bytes, void* stream);

/* Device status of the last wp_grid_batch(_fused) on batch_workspace (synchronizes `stream`):
   0, or WP_ERR_TIMEOUT when a gridding item's wait expired (fused form only). */
int wp_grid_batch_status(const void* batch_workspace, int32_t* status_host, void* stream);

/*
 * Self-test of the fused batch's failure path: the same launch with the scatter withheld and a
 * ~10 ms wait budget, so that every gridding item's wait expires; writes the resulting status
 * to *status_host (expected WP_ERR_TIMEOUT) and synchronizes.  No grid cell is written, nothing
 * faults or hangs, and the context stays usable.
 */
int wp_grid_batch_selftest(int32_t n_jobs, const wp_grid_job* jobs, void* batch_workspace,
                           size_t batch_workspace_bytes, int32_t* status_host, void* stream);

/* ---- differentiation of the visibility prediction ----------------------------------
 * Model: V = wp_degrid(K(t), wp_image_to_grid(I; t)) for a model image I and the radial
 * taper t, where the kernels K(t) come from wp_hankel_radial + wp_resample (supports and
 * plane values fixed).  For a real loss L the incoming gradient is g = dL/dRe V + j dL/dIm V
 * and complex gradients are returned in the same form (dL = Re(conj(gz) dz)).  The image
 * gradient is wp_dirty_image of wp_grid(g) (unit weights); the taper gradient is the sum of
 * wp_hankel_adjoint (kernels) and wp_image_adjoint (the division by t in the image step).
 */

/* Bytes of scratch for wp_grad_radial (the gridding workspace plus work-item lists). */
size_t wp_grad_workspace_bytes(const wp_plan* plan, int32_t P, int64_t V);

/*
 * Gradient of L with respect to the radial lines and their spline second derivatives:
 * for every visibility and every tap inside the support, Q = conj(g) G(cell) (w >= 0) or
 * g conj(G(cell)) (w < 0), spread onto the radial samples through the resample weights.
 *   grad_vis [V] complex (g), grid [N][N] complex (the grid that was degridded);
 *   grad_radial, grad_spline_m [P][K_out] complex out (overwritten; grad_spline_m may be
 *   NULL for linear interpolation).
 */
int wp_grad_radial(const wp_plan* plan, const wp_wkernels* kernels, const float* uvw,
                   const float* grad_vis, const float* grid, int64_t V, void* workspace,
                   size_t workspace_bytes, float* grad_radial, float* grad_spline_m, void* stream);

/*
 * Adjoint of kernel generation back to the taper (Section 4.3's transform is linear, so its
 * adjoint is the same matrix transposed): spline adjoint, dF = dC H, then
 * grad_taper[i] += sum_p Re(conj(dF_p,i) exp(+2 pi j w_p (n_i - 1))).
 *   workspace: the kernel-generation workspace prepared by wp_kernelgen_prepare;
 *   grad_taper [R] float, ACCUMULATED into.
 * Matrix routes only: a plan with kernelgen == WP_KG_PROJSLICE returns WP_ERR_UNSUPPORTED.
 */
int wp_hankel_adjoint(const wp_plan* plan, const double* w_planes, int32_t P, void* workspace,
                      size_t workspace_bytes, const float* grad_radial, const float* grad_spline_m,
                      float* grad_taper, void* stream);

/*
 * Image-side adjoint: with U = Re(centred inverse transform of grid_g) (grid_g = wp_grid of g
 * with unit weights; transformed in place), inside the circle
 *   grad_image = U / (t(r) weight_sum),  grad_taper += spread of -U I / (t(r)^2 weight_sum)
 * onto the taper nodes by the linear-interpolation weights; grad_image = 0 outside.
 */
int wp_image_adjoint(const wp_plan* plan, const float* taper, const float* image, float* grid_g,
                     double weight_sum, float* grad_image, float* grad_taper, void* stream);

/* ---- image <-> grid (Section 3: inverse transform and anti-aliasing correction) ----- */

/*
 * Dirty image from a grid:
 *   image[m][l] = Re sum_{v,u} grid[v][u] exp(+2 pi j ((u - N/2)(l - N/2) + (v - N/2)(m - N/2)) / N)
 *                 / (t(r) * weight_sum)    inside the circle (l - N/2)^2 + (m - N/2)^2 <= (N/2)^2,
 *   image = 0 outside it (Section 6: the Hankel image is valid in that circle), where
 *   t(r) is the taper linearly interpolated between its nodes r_i (clamped at the end
 *   nodes), r = dl sqrt((l - N/2)^2 + (m - N/2)^2).
 *   taper [R] float; grid [N][N] complex, OVERWRITTEN (transformed in place);
 *   image [N][N] float out.  Uses a cached cuFFT plan.
 */
int wp_dirty_image(const wp_plan* plan, const float* taper, float* grid, double weight_sum,
                   float* image, void* stream);

/*
 * wp_dirty_image normalised by a weight sum that stays on the device: weight_sum_dev points to
 * one device double -- normally stats[0] as accumulated by wp_grid, the sum of the weights of
 * the visibilities actually gridded (dropped ones and non-unit weights accounted for; Section 3:
 * the dirty image is the weighted mean of the gridded data).  The sum is read by the kernel, so
 * the call needs no host read-back and can follow wp_grid inside a captured stream.  A sum
 * <= 0 (nothing gridded) gives an all-zero image.  weight_sum_dev must be 8-byte aligned
 * (WP_ERR_SIZE otherwise); other arguments as wp_dirty_image.
 */
int wp_dirty_image_stats(const wp_plan* plan, const float* taper, float* grid,
                         const double* weight_sum_dev, float* image, void* stream);

/*
 * Adjoint of wp_dirty_image's linear map (without taking the real part), used to
 * predict visibilities of a model image with wp_degrid:
 *   grid[v][u] = sum_{m,l inside circle} image[m][l] / (t(r) weight_sum)
 *                exp(-2 pi j ((u - N/2)(l - N/2) + (v - N/2)(m - N/2)) / N)
 *   image [N][N] float in; grid [N][N] complex out (overwritten).
 */
int wp_image_to_grid(const wp_plan* plan, const float* taper, const float* image,
                     double weight_sum, float* grid, void* stream);

/* ---- measurement --------------------------------------------------------------------- */

/*
 * Measurement helper with no counterpart in the paper: queues one launch of blocks_per_sm
 * blocks per SM of 256 threads, each thread running eight independent register-resident FP32
 * FMA chains for 16 * iters steps, and writes to *flops_out (host) the FLOP count of that launch
 * (2 per FMA).  Timing it with CUDA events on `stream` gives the device's FP32 FMA rate -- the
 * denominator of the gridder's ALU roofline.  sink: one device float, written only in a case
 * the chains never reach.  WP_ERR_SIZE for iters < 1 or blocks_per_sm outside 1..64.
 */
int wp_probe_fp32_fma(int32_t iters, int32_t blocks_per_sm, float* sink, double* flops_out,
                      void* stream);

/*
 * Measurement helper with no counterpart in the paper: queues one launch of blocks_per_sm blocks
 * per SM of 256 threads in which every warp, steps times, reads ten rows of 32 consecutive
 * complex64 values at a pseudo-random position of buf, the rows W values apart -- the shape of
 * the slot gridder's tap loads (one 8-byte load per lane per row of a sub-kernel) -- and writes
 * to *bytes_out (host) the bytes that launch reads.  Timed with CUDA events on `stream`, it gives
 * the rate at which L2 serves that pattern when buf (n_elems complex64, device memory, 8-byte
 * aligned) fits in L2: the denominator of the gridder's L2 roofline.  sink: one device float,
 * written only in a case the loads never reach.  WP_ERR_SIZE for W outside 1..4096, steps < 1,
 * blocks_per_sm outside 1..64, an unaligned buf, or n_elems not above 9 W + 32 or more than
 * 2^32 above it.
 */
int wp_probe_l2_taps(const void* buf, int64_t n_elems, int32_t W, int32_t steps, int32_t blocks_per_sm,
                     float* sink, double* bytes_out, void* stream);

/* ---- checked build ------------------------------------------------------------------- */

/*
 * A stand-in for a memory checker, with no counterpart in the paper.  The library compiled with
 * -DWP_CHECK_BOUNDS (paper_1904_08463_gb300.build.build_checked) tests the index of every tap
 * read and grid cell access of the gridders (grid_method 3 and 9, per call and batched), the
 * degridders (0 and 9) and every kernel-cache row the resample writes, against the extent of
 * its buffer: the plane's block [offsets[p], offsets[p+1]) of the cache, the N x N grid, the V
 * visibilities.  An access outside is skipped, and the first one of each translation unit is
 * recorded as site << 48 | (index & 0xffffffffffff), sites 1 cache row written, 2 tap read,
 * 3 grid cell, 4 visibility written.  wp_bounds_status synchronizes the device, writes to
 * *first (host) the first record found (0: none) and clears the records when clear != 0.
 * The default build keeps no checks and returns WP_ERR_UNSUPPORTED.
 */
int wp_bounds_status(uint64_t* first, int32_t clear);

/* ---- misc ---------------------------------------------------------------------------- */
const char* wp_strerror(int code);
const char* wp_last_error_string(void);   /* last CUDA/cuFFT error text (thread-local) */
int wp_version(void);                      /* major*10000 + minor*100 + patch           */
void wp_release(void);                     /* free cached cuFFT plans of this process   */

#ifdef __cplusplus
}
#endif
#endif /* WPROJ_H */
