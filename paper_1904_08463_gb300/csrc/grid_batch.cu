// Persistent gridding of many independent problems in one launch (batched uneven imaging
// problems; Alg. 1 / Alg. 2 gridding step for each problem).
//
// Per job the binning runs as for wp_grid up to the list of live work items (FP64 decisions,
// bin counts and their scan, item flags and their scan, the item list) -- but not the scatter
// of the records into bin order.  Then ONE persistent launch takes work from a single device
// queue: first the scatter chunks of every job (SCATTER_CHUNK visibilities each), then the
// (plane, output tile) gridding items of every job, largest jobs first as the caller ordered
// them.  A gridding item of job j reads the bin-ordered records that job j's scatter chunks
// write in the same launch, so its block first waits until all of them are done: a counter per
// job that every finished chunk increments after a fence.  The queue hands out work in order,
// so every chunk a gridding item waits for was taken earlier by a block that is running and
// waits for nothing -- the wait always ends; it is nevertheless bounded by a clock budget,
// after which the item is skipped and WP_ERR_TIMEOUT recorded in the batch status.  Small jobs'
// items fill the GPU beside large ones', with no tail per job and one launch for the batch.
#include <cuda_runtime.h>

#include <vector>

#include "wp_internal.cuh"
#include "grid_ro.cuh"
#include "grid_slot.cuh"

namespace wp {

namespace {
constexpr int SCATTER_CHUNK = GRID_WARPS * 32 * 8;   // visibilities per scatter work item
constexpr long long WAIT_BUDGET = 1LL << 31;         // SM clock cycles (~1 s)
}  // namespace

struct BatchJob {
    int mode;                                 // 3: row-owned tiles, 9: slots
    int P;
    int N, os, s_max, ntx, ntiles, n_sc;      // n_sc: producer chunks of the job (scatter or gather)
    int64_t V;
    const int32_t* seff;
    const int64_t* offsets;
    const float2* cache;
    const int* start;                         // bin starts (scanned counts)
    const int* key;                           // bin key per visibility, -1 when dropped
    const int4* rec;
    const float2* vis;
    const float* weight;
    int* cursor;
    int4* srec;
    float2* svis;
    const int* items;
    const int* ctrl;                          // ctrl[1]: number of live items (row-owned)
    float2* grid;
    const int* vstart;                        // slots: plane bounds of the sorted list,
    const int* istart;                        //        item starts per plane (istart[P] = items),
    const uint32_t* sidx;                     //        the sort's permutation
};

struct BatchTable {
    BatchJob j[WP_GRID_BATCH_MAX_JOBS];
};

// ctrl layout: [0] queue head, [1] status, [2 .. 2 + n_jobs) finished scatter chunks per job
// HAS_RO / HAS_SLOT: which kinds of job the batch holds (the row-owned tile's shared memory and
// the slot code's registers are only paid for when used).
template <int TILE, bool HAS_RO, bool HAS_SLOT>
__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid_batch(const __grid_constant__ BatchTable tab, int n_jobs,
                                                                int* __restrict__ bctrl, long long budget,
                                                                int withhold_scatter) {
    static_assert(SLOT_WARPS == GRID_WARPS, "a slot unit is one item per warp of the block");
    __shared__ float2 tile[HAS_RO ? TILE * TILE : 1];
    __shared__ int l_off[RO_LIST];
    __shared__ uint32_t l_geo[RO_LIST];
    __shared__ float2 l_vv[RO_LIST];
    __shared__ int s_idx, s_n, s_ok;
    __shared__ int pre_sc[WP_GRID_BATCH_MAX_JOBS + 1];   // prefix of scatter chunks
    __shared__ int pre_gi[WP_GRID_BATCH_MAX_JOBS + 1];   // prefix of gridding items
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int k = 0; k < n_jobs; ++k) {
            pre_sc[k] = a;
            pre_gi[k] = b;
            a += tab.j[k].n_sc;
            // consumer units: one row-owned item, or one slot item per warp of the block
            b += (tab.j[k].mode == 9) ? (tab.j[k].istart[tab.j[k].P] + SLOT_WARPS - 1) / SLOT_WARPS
                                      : tab.j[k].ctrl[1];
        }
        pre_sc[n_jobs] = a;
        pre_gi[n_jobs] = b;
    }
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) tile[i] = make_float2(0.0f, 0.0f);
    __syncthreads();
    const int n_sc = pre_sc[n_jobs], n_gi = pre_gi[n_jobs];
    int* status = bctrl + 1;
    int* done = bctrl + 2;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&bctrl[0], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n_sc + n_gi) break;
        if (idx < n_sc) {
            // ---- scatter chunk: records and weighted values into bin order
            int jb = 0;
            while (jb + 1 < n_jobs && pre_sc[jb + 1] <= idx) ++jb;
            const BatchJob& J = tab.j[jb];
            if (withhold_scatter) continue;       // self-test: the chunk is never done
            const int64_t k0 = (int64_t)(idx - pre_sc[jb]) * SCATTER_CHUNK;
            if (HAS_SLOT && J.mode == 9) {
                // gather: sorted position i takes its record and weighted value
                const int64_t n_kept = J.vstart[J.P];
                for (int64_t i = k0 + threadIdx.x; i < min(n_kept, k0 + SCATTER_CHUNK); i += blockDim.x)
                    slot_gather_one(i, J.os, J.s_max, J.sidx, J.rec, J.seff, J.vis, J.weight, J.srec, J.svis);
            } else if (HAS_RO) {
                for (int64_t k = k0 + threadIdx.x; k < min(J.V, k0 + SCATTER_CHUNK); k += blockDim.x) {
                    const int kk = J.key[k];
                    if (kk < 0) continue;
                    const int pos = J.start[kk] + atomicAdd(&J.cursor[kk], 1);
                    J.srec[pos] = J.rec[k];
                    const float2 v = J.vis[k];
                    const float a = J.weight ? J.weight[k] : 1.0f;
                    J.svis[pos] = make_float2(v.x * a, v.y * a);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();                  // the chunk's writes before its count
                atomicAdd(&done[jb], 1);
            }
        } else {
            // ---- gridding item: wait (bounded) for the job's scatter, then the row-owned tile
            const int g = idx - n_sc;
            int jb = 0;
            while (jb + 1 < n_jobs && pre_gi[jb + 1] <= g) ++jb;
            const BatchJob& J = tab.j[jb];
            if (threadIdx.x == 0) {
                int ok = 1;
                const long long t0 = clock64();
                while (atomicAdd(&done[jb], 0) < J.n_sc) {
                    // after one expiry the batch has failed: later items give up at once
                    if (clock64() - t0 > budget || atomicAdd(status, 0) != 0) {
                        atomicMin(status, WP_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();                  // the job's records after its count
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) continue;
            if (HAS_SLOT && J.mode == 9) {
                const int it = (g - pre_gi[jb]) * SLOT_WARPS + (int)(threadIdx.x >> 5);
                if (it < J.istart[J.P])
                    slot_item<SLOT_ROWS, true>(it, J.N, J.P, J.s_max, J.seff, J.offsets, J.cache, J.vstart,
                                               J.istart, J.srec, J.svis, J.grid);
            } else if (HAS_RO) {
                const int item = J.items[g - pre_gi[jb]];
                ro_item<TILE, true>(item, J.N, J.os, J.s_max, J.ntx, J.ntiles, J.seff, J.offsets, J.cache, J.start,
                                    J.srec, J.svis, J.grid, tile, l_off, l_geo, l_vv, &s_n);
            }
        }
    }
}

// Item list from the in-place scan of the flags (n + 1 entries, pos[n] = total): item it is live
// when pos[it + 1] > pos[it].  Leaves the cursor array free for the scatter.
__global__ void __launch_bounds__(256) k_item_write_pos(int64_t n, const int* __restrict__ pos,
                                                        int* __restrict__ items, int* __restrict__ ctrl) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it < n && pos[it + 1] > pos[it]) items[pos[it]] = (int)it;
    if (it == n - 1) ctrl[1] = pos[n];
}

size_t grid_batch_ctrl_bytes() { return (size_t)(2 + WP_GRID_BATCH_MAX_JOBS) * sizeof(int) + 256; }

// Binning of one job up to its item list (no scatter); the batch kernel scatters.
int grid_batch_prepare(const Geom& g, const wp_wkernels* kern, const float* uvw, const float* weight, int64_t V,
                       const GridWork& w, cudaStream_t st) {
    int rc = grid_bin_noscatter(g, kern, uvw, weight, V, w, st);
    if (rc) return rc;
    const int64_t n = (int64_t)kern->P * w.ntiles;
    rc = item_flags(g, kern, w, st);
    if (rc) return rc;
    rc = exclusive_scan_i32(w.flags, w.flags, n + 1, w.scan_tmp, st);
    if (rc) return rc;
    k_item_write_pos<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, w.flags, w.items, w.ctrl);
    WP_LAUNCH_CHECK("k_item_write_pos");
    return WP_OK;
}

int grid_batch_run(int n_jobs, const Geom* geoms, const wp_wkernels* kerns, const float* const* vis,
                   const float* const* weight, const int64_t* Vs, const GridWork* works, float* const* grids,
                   const uint32_t* const* sidx, int tile, void* bws, long long budget, int withhold, cudaStream_t st) {
    BatchTable tab;
    bool has_ro = false, has_slot = false;
    for (int k = 0; k < n_jobs; ++k) {
        BatchJob& J = tab.j[k];
        const GridWork& w = works[k];
        J.mode = (geoms[k].grid_method == 9) ? 9 : 3;
        (J.mode == 9 ? has_slot : has_ro) = true;
        J.P = kerns[k].P;
        J.vstart = w.vstart;
        J.istart = w.istart;
        J.sidx = sidx[k];
        J.N = geoms[k].N;
        J.os = geoms[k].os;
        J.s_max = geoms[k].s_max;
        J.ntx = w.ntx;
        J.ntiles = w.ntiles;
        J.V = Vs[k];
        J.n_sc = (int)((Vs[k] + SCATTER_CHUNK - 1) / SCATTER_CHUNK);
        J.seff = w.seff;
        J.offsets = kerns[k].offsets;
        J.cache = reinterpret_cast<const float2*>(kerns[k].cache);
        J.start = w.count;
        J.key = w.key;
        J.rec = w.rec;
        J.vis = reinterpret_cast<const float2*>(vis[k]);
        J.weight = weight[k];
        J.cursor = w.cursor;
        J.srec = w.srec;
        J.svis = w.svis;
        J.items = w.items;
        J.ctrl = w.ctrl;
        J.grid = reinterpret_cast<float2*>(grids[k]);
    }
    int* bctrl = static_cast<int*>(bws);
    WP_CUDA(cudaMemsetAsync(bctrl, 0, (size_t)(2 + n_jobs) * sizeof(int), st));
    int dev = 0, sms = 0, per_sm = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
#define WP_LAUNCH_BATCH(T, R, S)                                                                               \
    do {                                                                                                       \
        WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_batch<T, R, S>, GRID_WARPS * 32, 0)); \
        if (per_sm < 1) per_sm = 1;                                                                            \
        k_grid_batch<T, R, S><<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(tab, n_jobs, bctrl, budget, withhold); \
    } while (0)
    if (!has_ro) WP_LAUNCH_BATCH(64, false, true);
    else if (tile == 32) { if (has_slot) WP_LAUNCH_BATCH(32, true, true); else WP_LAUNCH_BATCH(32, true, false); }
    else { if (has_slot) WP_LAUNCH_BATCH(64, true, true); else WP_LAUNCH_BATCH(64, true, false); }
#undef WP_LAUNCH_BATCH
    WP_LAUNCH_CHECK("k_grid_batch");
    return WP_OK;
}

long long grid_batch_budget() { return WAIT_BUDGET; }

}  // namespace wp

using namespace wp;

namespace {
int batch_call(int32_t n_jobs, const wp_grid_job* jobs, void* bws, size_t bws_bytes, long long budget, int withhold,
               cudaStream_t st) {
    if (n_jobs < 1 || n_jobs > WP_GRID_BATCH_MAX_JOBS) return WP_ERR_SIZE;
    if (!jobs || !bws) return WP_ERR_NULL;
    if (((uintptr_t)bws & 255u) || bws_bytes < grid_batch_ctrl_bytes()) return WP_ERR_WORKSPACE;
    int tile = 0;                                    // the row-owned jobs' tile (all the same)
    for (int k = 0; k < n_jobs; ++k)
        if (jobs[k].plan.grid_method != 9) {
            tile = jobs[k].plan.grid_tile ? jobs[k].plan.grid_tile : 64;
            break;
        }
    std::vector<Geom> geoms((size_t)n_jobs);
    std::vector<GridWork> works((size_t)n_jobs);
    std::vector<wp_wkernels> kerns((size_t)n_jobs);
    std::vector<const float*> vis((size_t)n_jobs), weight((size_t)n_jobs);
    std::vector<int64_t> Vs((size_t)n_jobs);
    std::vector<float*> grids((size_t)n_jobs);
    for (int k = 0; k < n_jobs; ++k) {               // every job checked before any launch
        const wp_grid_job& J = jobs[k];
        wp_plan plan = J.plan;
        if (plan.grid_method != 9) {
            if ((plan.grid_tile ? plan.grid_tile : 64) != tile) return WP_ERR_PLAN;
            plan.grid_method = 3;
        }
        int rc = check_grid_args(&plan, &J.kernels, J.uvw, J.V, J.workspace, J.workspace_bytes, &geoms[(size_t)k],
                                 true);
        if (rc) return rc;
        if (!J.grid || (J.V > 0 && !J.vis)) return WP_ERR_NULL;
        carve_grid(geoms[(size_t)k], J.kernels.P, J.V, J.workspace, J.workspace_bytes, &works[(size_t)k]);
        kerns[(size_t)k] = J.kernels;
        vis[(size_t)k] = J.vis;
        weight[(size_t)k] = J.weight;
        Vs[(size_t)k] = J.V;
        grids[(size_t)k] = J.grid;
    }
    std::vector<const uint32_t*> sidx((size_t)n_jobs, nullptr);
    for (int k = 0; k < n_jobs; ++k) {
        const Geom& g = geoms[(size_t)k];
        int rc = (g.grid_method == 9)
                     ? grid_slot_prepare(g, &kerns[(size_t)k], jobs[k].uvw, jobs[k].weight, jobs[k].V, works[(size_t)k],
                                         st, &sidx[(size_t)k])
                     : grid_batch_prepare(g, &kerns[(size_t)k], jobs[k].uvw, jobs[k].weight, jobs[k].V,
                                          works[(size_t)k], st);
        if (rc) return rc;
    }
    int rc = grid_batch_run(n_jobs, geoms.data(), kerns.data(), vis.data(), weight.data(), Vs.data(), works.data(),
                            grids.data(), sidx.data(), tile ? tile : 64, bws, budget, withhold, st);
    if (rc) return rc;
    if (!withhold)
        for (int k = 0; k < n_jobs; ++k)
            if (jobs[k].stats && (rc = add_stats(jobs[k].stats, works[(size_t)k].red, st))) return rc;
    return WP_OK;
}
}  // namespace

extern "C" {

size_t wp_grid_batch_workspace_bytes(void) { return grid_batch_ctrl_bytes(); }

int wp_grid_batch(int32_t n_jobs, const wp_grid_job* jobs, void* batch_workspace, size_t batch_workspace_bytes,
                  void* stream) {
    WP_RANGE("wp_grid_batch");
    return batch_call(n_jobs, jobs, batch_workspace, batch_workspace_bytes, grid_batch_budget(), 0,
                      (cudaStream_t)stream);
}

int wp_grid_batch_status(const void* batch_workspace, int32_t* status_host, void* stream) {
    if (!batch_workspace || !status_host) return WP_ERR_NULL;
    const int* bctrl = static_cast<const int*>(batch_workspace);
    WP_CUDA(cudaMemcpyAsync(status_host, bctrl + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    WP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return WP_OK;
}

int wp_grid_batch_selftest(int32_t n_jobs, const wp_grid_job* jobs, void* batch_workspace,
                           size_t batch_workspace_bytes, int32_t* status_host, void* stream) {
    WP_RANGE("wp_grid_batch_selftest");
    if (!status_host) return WP_ERR_NULL;
    // scatter withheld, 2e7-cycle (~10 ms) budget: every gridding item's wait expires
    int rc = batch_call(n_jobs, jobs, batch_workspace, batch_workspace_bytes, 20000000LL, 1, (cudaStream_t)stream);
    if (rc) return rc;
    return wp_grid_batch_status(batch_workspace, status_host, stream);
}

}  // extern "C"
