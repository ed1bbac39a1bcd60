// Persistent gridding of many independent problems (batched uneven imaging problems; Alg. 1 /
// Alg. 2 gridding step for each problem).
//
// Per job the binning runs as for wp_grid up to the list of live work items (FP64 decisions,
// bin counts and their scan, item flags and their scan, the item list) -- but not the scatter
// of the records into bin order (the gather into sorted order for slot jobs).  Then persistent
// launches take work from one device queue per gridder kind: the producer chunks of every job
// (scatter or gather, SCATTER_CHUNK / SLOT_GATHER records each) and the gridding items of every
// job ((plane, output tile) blocks, or slot tiles per warp), largest jobs first as the caller
// ordered them; small jobs' items fill the GPU beside large ones', with no tail per job.
//
// Two forms.  Default (wp_grid_batch): per kind, one launch that runs the producer chunks of
// every job and a second that runs the items of every job, which read the ordered records
// through the read-only path.  Fused (wp_grid_batch_fused): per kind, ONE launch whose queue
// holds each job's producer chunks right before its items, job after job; a gridding item of
// job j reads the records that job j's producer chunks write in the same launch, so it first
// waits until all of them are done: a counter per job that every finished chunk increments after
// a fence.  The queue hands out work in order, so every chunk an item waits for was taken earlier
// by a block that is running and waits for nothing -- the wait always ends; it is nevertheless
// bounded by a clock budget, after which the item is skipped and WP_ERR_TIMEOUT recorded in the
// batch status.  On 48 problems (one GB300) the default form takes 278-283 ms per call, the fused
// one 289-294 ms (300 ms with every job's chunks ahead of every job's items), both above the
// 250-253 ms of the same jobs gridded one wp_grid call at a time.
#include <cuda_runtime.h>

#include <vector>

#include "wp_internal.cuh"
#include "grid_ro.cuh"
#include "grid_slot.cuh"

namespace wp {

namespace {
constexpr int SCATTER_CHUNK = GRID_WARPS * 32 * 8;   // visibilities per scatter work item
constexpr long long WAIT_BUDGET = 1LL << 31;         // SM clock cycles (~1 s)
// batch control words: [0] row-owned queue head, [1] status, [2 .. 2 + MAX) finished producer
// chunks per job, [2 + MAX] slot queue head, [BATCH_PRE ..) the four job prefixes
constexpr int BATCH_PRE = 3 + WP_GRID_BATCH_MAX_JOBS + 2;
constexpr int HEAD2_RO = 3 + WP_GRID_BATCH_MAX_JOBS, HEAD2_SLOT = 4 + WP_GRID_BATCH_MAX_JOBS;
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

// Bounded wait (one thread) until *done reaches `need` producer chunks; false -- with
// WP_ERR_TIMEOUT recorded -- once the clock budget runs out or another wait already failed.
// The acquire fence orders the job's records after its count.
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Polls with plain acquire loads (no read-modify-write: hundreds of blocks polling one counter
// must not queue at its L2 slice ahead of the producers' increments) and backs off from 64 ns
// to 4 us between polls.
__device__ __forceinline__ int wait_done(int* done, int need, int* status, long long budget) {
    if (ld_acquire(done) >= need) return 1;
    int ok = 1;
    unsigned ns = 64;
    const long long t0 = clock64();
    while (ld_acquire(done) < need) {
        if (clock64() - t0 > budget || ld_acquire(status) != 0) {
            atomicMin(status, WP_ERR_TIMEOUT);
            ok = 0;
            break;
        }
        __nanosleep(ns);
        ns = ns < 4096 ? 2 * ns : 4096;
    }
    __threadfence();
    return ok;
}

// ctrl layout: [0] queue head, [1] status, [2 .. 2 + n_jobs) finished scatter chunks per job
// Job prefixes of both kernels' queues, once per batch (one warp): producer chunks and gridding
// work of every job, counted where the binning left them on the device.  Layout after the
// counters: pre[0 .. 6][n_jobs + 1] = row-owned chunks, row-owned items, slot chunks, slot items,
// row-owned chunks + items, slot chunks + items (the fused form's queue: each job's producer
// chunks right before its items).
constexpr int SLOT_GATHER = 32 * 32;     // sorted positions per gather work unit (one warp)

__global__ void k_batch_prefix(const __grid_constant__ BatchTable tab, int n_jobs, int* __restrict__ pre) {
    if (threadIdx.x != 0) return;
    int a = 0, b = 0, c = 0, d = 0;
    for (int k = 0; k <= n_jobs; ++k) {
        pre[k] = a;
        pre[(n_jobs + 1) + k] = b;
        pre[2 * (n_jobs + 1) + k] = c;
        pre[3 * (n_jobs + 1) + k] = d;
        pre[4 * (n_jobs + 1) + k] = a + b;
        pre[5 * (n_jobs + 1) + k] = c + d;
        if (k == n_jobs) break;
        const BatchJob& J = tab.j[k];
        if (J.mode == 9) {
            c += (int)((J.V + SLOT_GATHER - 1) / SLOT_GATHER);
            d += J.istart[J.P];
        } else {
            a += J.n_sc;
            b += J.ctrl[1];
        }
    }
}

// largest k in [0, n_jobs) with pre[k] <= idx (pre ascending, pre[0] = 0 <= idx)
__device__ __forceinline__ int job_of(const int* __restrict__ pre, int n_jobs, int idx) {
    int lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= idx) lo = mid; else hi = mid;
    }
    return lo;
}

// Queue position idx -> (job jb, producer chunk or item `loc` of that job); true for a producer
// chunk.  Fused form (phase 0): each job's chunks then its items, job after job (pre_cb); the
// split forms: every job's chunks (pre_sc), then every job's items (pre_gi).
__device__ __forceinline__ bool batch_decode(int phase, int idx, int n_jobs, int n_sc, const int* __restrict__ pre_sc,
                                             const int* __restrict__ pre_gi, const int* __restrict__ pre_cb, int& jb,
                                             int& loc) {
    if (phase == 0) {
        jb = job_of(pre_cb, n_jobs, idx);
        loc = idx - __ldg(pre_cb + jb);
        const int ns = __ldg(pre_sc + jb + 1) - __ldg(pre_sc + jb);
        if (loc < ns) return true;
        loc -= ns;
        return false;
    }
    if (idx < n_sc) {
        jb = job_of(pre_sc, n_jobs, idx);
        loc = idx - __ldg(pre_sc + jb);
        return true;
    }
    jb = job_of(pre_gi, n_jobs, idx - n_sc);
    loc = idx - n_sc - __ldg(pre_gi + jb);
    return false;
}

// Row-owned jobs: block-level work (a scatter chunk, or one (plane, tile) item per block).
template <int TILE>
__global__ void __launch_bounds__(GRID_WARPS * 32, 6) k_grid_batch_ro(const __grid_constant__ BatchTable tab, int n_jobs,
                                                                   int* __restrict__ bctrl, long long budget,
                                                                   int withhold_scatter, int phase) {
    __shared__ float2 tile[TILE * TILE];
    __shared__ int l_off[RO_LIST];
    __shared__ uint32_t l_geo[RO_LIST];
    __shared__ float2 l_vv[RO_LIST];
    __shared__ int s_idx, s_n, s_ok;
    const int* pre_sc = bctrl + BATCH_PRE;                    // prefix of scatter chunks
    const int* pre_gi = pre_sc + (n_jobs + 1);                // prefix of gridding items
    const int* pre_cb = pre_sc + 4 * (n_jobs + 1);            // prefix of both (fused queue)
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) tile[i] = make_float2(0.0f, 0.0f);
    __syncthreads();
    const int n_sc = pre_sc[n_jobs], n_gi = pre_gi[n_jobs];
    int* status = bctrl + 1;
    int* done = bctrl + 2;
    for (;;) {
        if (threadIdx.x == 0) s_idx = (phase == 2) ? n_sc + atomicAdd(&bctrl[HEAD2_RO], 1) : atomicAdd(&bctrl[0], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= (phase == 1 ? n_sc : n_sc + n_gi)) break;
        int jb, loc;
        const bool prod = batch_decode(phase, idx, n_jobs, n_sc, pre_sc, pre_gi, pre_cb, jb, loc);
        if (prod) {
            // ---- scatter chunk: records and weighted values into bin order
            const BatchJob& J = tab.j[jb];
            if (withhold_scatter) continue;       // self-test: the chunk is never done
            const int64_t k0 = (int64_t)loc * SCATTER_CHUNK;
            for (int64_t k = k0 + threadIdx.x; k < min(J.V, k0 + SCATTER_CHUNK); k += blockDim.x) {
                const int kk = J.key[k];
                if (kk < 0) continue;
                const int pos = J.start[kk] + atomicAdd(&J.cursor[kk], 1);
                J.srec[pos] = J.rec[k];
                const float2 v = J.vis[k];
                const float a = J.weight ? J.weight[k] : 1.0f;
                J.svis[pos] = make_float2(v.x * a, v.y * a);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();                  // the chunk's writes before its count
                atomicAdd(&done[jb], 1);
            }
        } else {
            // ---- gridding item: wait (bounded) for the job's scatter, then the row-owned tile
            const BatchJob& J = tab.j[jb];
            const int item = J.items[loc];
            if (phase == 2) {
                ro_item<TILE, false>(item, J.N, J.os, J.s_max, J.ntx, J.ntiles, J.seff, J.offsets, J.cache, J.start,
                                     J.srec, J.svis, J.grid, tile, l_off, l_geo, l_vv, &s_n);
                continue;
            }
            if (threadIdx.x == 0) s_ok = wait_done(&done[jb], J.n_sc, status, budget);
            __syncthreads();
            if (!s_ok) continue;
            ro_item<TILE, true>(item, J.N, J.os, J.s_max, J.ntx, J.ntiles, J.seff, J.offsets, J.cache, J.start,
                                J.srec, J.svis, J.grid, tile, l_off, l_geo, l_vv, &s_n);
        }
    }
}

// Slot jobs: warp-level work from the same kind of queue -- a gather chunk (SLOT_GATHER sorted
// positions), or one slot item -- so that no warp waits for the others of its block.

__global__ void __launch_bounds__(SLOT_WARPS * 32, 3) k_grid_batch_slot(const __grid_constant__ BatchTable tab,
                                                                        int n_jobs, int* __restrict__ bctrl,
                                                                        long long budget, int withhold_gather,
                                                                        int phase) {
    const int* pre_sc = bctrl + BATCH_PRE + 2 * (n_jobs + 1);  // prefix of gather chunks
    const int* pre_gi = pre_sc + (n_jobs + 1);                // prefix of slot items
    const int* pre_cb = pre_sc + 3 * (n_jobs + 1);            // prefix of both (fused queue)
    const int lane = threadIdx.x & 31;
    const int n_sc = pre_sc[n_jobs], n_gi = pre_gi[n_jobs];
    int* head = bctrl + 2 + WP_GRID_BATCH_MAX_JOBS;
    int* status = bctrl + 1;
    int* done = bctrl + 2;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = (phase == 2) ? n_sc + atomicAdd(&bctrl[HEAD2_SLOT], 1) : atomicAdd(head, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= (phase == 1 ? n_sc : n_sc + n_gi)) break;
        int jb, loc;
        const bool prod = batch_decode(phase, idx, n_jobs, n_sc, pre_sc, pre_gi, pre_cb, jb, loc);
        if (prod) {
            const BatchJob& J = tab.j[jb];
            if (withhold_gather) continue;        // self-test: the chunk is never done
            const int64_t i0 = (int64_t)loc * SLOT_GATHER;
            const int64_t n_kept = J.vstart[J.P];
            for (int64_t i = i0 + lane; i < min(n_kept, i0 + SLOT_GATHER); i += 32)
                slot_gather_one(i, J.os, J.s_max, J.sidx, J.rec, J.seff, J.vis, J.weight, J.srec, J.svis);
            __syncwarp();
            if (lane == 0) {
                __threadfence();                  // the chunk's writes before its count
                atomicAdd(&done[jb], 1);
            }
        } else {
            const BatchJob J = tab.j[jb];   // copied once per item: 3 % faster than reading the table in the walk
            if (phase == 2) {
                slot_item<SLOT_ROWS, false, false, true>(loc, J.N, J.P, J.s_max, J.seff, J.offsets, J.cache, J.vstart,
                                            J.istart, J.srec, J.svis, J.grid);
                continue;
            }
            int ok = 0;
            if (lane == 0) ok = wait_done(&done[jb], (int)((J.V + SLOT_GATHER - 1) / SLOT_GATHER), status, budget);
            if (!__shfl_sync(0xffffffffu, ok, 0)) continue;
            slot_item<SLOT_ROWS, true, false, true>(loc, J.N, J.P, J.s_max, J.seff, J.offsets, J.cache, J.vstart,
                                       J.istart, J.srec, J.svis, J.grid);
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

size_t grid_batch_ctrl_bytes() {
    return (size_t)(BATCH_PRE + 6 * (WP_GRID_BATCH_MAX_JOBS + 1)) * sizeof(int) + 256;
}

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
                   const uint32_t* const* sidx, int tile, void* bws, long long budget, int withhold, int fused,
                   cudaStream_t st) {
    // fused: one launch per gridder kind, items waiting (bounded) for their job's producers;
    // otherwise two: the producer chunks, then the items (records through the read-only path)
    const bool phased = !fused;
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
    WP_CUDA(cudaMemsetAsync(bctrl, 0, (size_t)BATCH_PRE * sizeof(int), st));
    k_batch_prefix<<<1, 32, 0, st>>>(tab, n_jobs, bctrl + BATCH_PRE);
    WP_LAUNCH_CHECK("k_batch_prefix");
    int dev = 0, sms = 0, per_sm = 0;
    WP_CUDA(cudaGetDevice(&dev));
    WP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the row-owned jobs first, then the slot jobs, each kernel with its own queue over its jobs
    if (has_ro) {
        auto kro = (tile == 32) ? k_grid_batch_ro<32> : k_grid_batch_ro<64>;
        WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kro, GRID_WARPS * 32, 0));
        if (per_sm < 1) per_sm = 1;
        for (int ph = phased ? 1 : 0; ph <= (phased ? 2 : 0); ++ph) {
            kro<<<sms * per_sm, GRID_WARPS * 32, 0, st>>>(tab, n_jobs, bctrl, budget, withhold, ph);
            WP_LAUNCH_CHECK("k_grid_batch_ro");
        }
    }
    if (has_slot) {
        WP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_batch_slot, SLOT_WARPS * 32, 0));
        if (per_sm < 1) per_sm = 1;
        for (int ph = phased ? 1 : 0; ph <= (phased ? 2 : 0); ++ph) {
            k_grid_batch_slot<<<sms * per_sm, SLOT_WARPS * 32, 0, st>>>(tab, n_jobs, bctrl, budget, withhold, ph);
            WP_LAUNCH_CHECK("k_grid_batch_slot");
        }
    }
    return WP_OK;
}

long long grid_batch_budget() { return WAIT_BUDGET; }

}  // namespace wp

using namespace wp;

namespace {
int batch_call(int32_t n_jobs, const wp_grid_job* jobs, void* bws, size_t bws_bytes, long long budget, int withhold,
               int fused, cudaStream_t st) {
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
                            grids.data(), sidx.data(), tile ? tile : 64, bws, budget, withhold, fused, st);
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
    return batch_call(n_jobs, jobs, batch_workspace, batch_workspace_bytes, grid_batch_budget(), 0, 0,
                      (cudaStream_t)stream);
}

int wp_grid_batch_fused(int32_t n_jobs, const wp_grid_job* jobs, void* batch_workspace, size_t batch_workspace_bytes,
                        void* stream) {
    WP_RANGE("wp_grid_batch_fused");
    return batch_call(n_jobs, jobs, batch_workspace, batch_workspace_bytes, grid_batch_budget(), 0, 1,
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
    int rc = batch_call(n_jobs, jobs, batch_workspace, batch_workspace_bytes, 20000000LL, 1, 1, (cudaStream_t)stream);
    if (rc) return rc;
    return wp_grid_batch_status(batch_workspace, status_host, stream);
}

}  // extern "C"
