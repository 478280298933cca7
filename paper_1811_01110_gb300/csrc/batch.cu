// batch.cu -- many plans in one persistent, load-balanced launch.
//
// The work items of every plan (each already cut by its own schedule) are
// merged into one queue, plan by plan (the plans with the most work first, so
// the smallest surfaces' light items fill the end), each plan's items heaviest
// first: a surface's sources then stay in L2 while its items run.  A
// persistent grid (one wave: the occupancy limit times the SM count) of
// independent warps pops items from the queue with an atomic counter, so a
// warp that finishes a light item immediately takes the next one; each item
// carries its plan index, and the order p may differ between plans (the item
// body is instantiated per p and selected per item; the batch always runs
// the per-order item bodies, whatever a plan's p_unroll).  In single-layer
// mixed batches up to four consecutive single-target items of one plan run
// together (8 or 16 lanes each), so that their dependent loads overlap, and
// four whose lists are single runs with a short union stage that union once
// (laplace_mixed_window4).  The whole sequence --
// copy of the per-evaluation pointer table, w mu preparation for every plan,
// queue reset, persistent kernel, slice combine -- is captured once into a
// CUDA graph and replayed per evaluation.
#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "laplace_items.cuh"
#include "plan_internal.h"

using namespace tsqbx;

namespace {

// Items a warp takes from the queue per atomic operation.
constexpr unsigned kPopChunk = 8;

struct BatchIO {
    const double *density;
    double *out_slp, *out_dlp;
};

struct BatchPlan {
    DevGeom g;
    DevEval ev;      // wmu, partial buffers and status owned by the batch
    int p;
};

struct BatchCombine {
    Combine c;
    int plan;
};

__global__ void batch_prep_kernel(const BatchPlan *plans, const BatchIO *io, int mixed)
{
    const BatchPlan &bp = plans[blockIdx.y];
    const double *mu = io[blockIdx.y].density;
    const int64_t n = bp.g.n_src;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = bp.g.src_pw[i].w * mu[i];
        if (mixed) const_cast<float *>(bp.ev.wmu_f)[i] = (float)v;
        else const_cast<double *>(bp.ev.wmu)[i] = v;
    }
}

// Where each queued item's slice starts in its plan's run lists.
__global__ void batch_walk_kernel(const BatchPlan *plans, const Item *items, int64_t n_items, WalkStart *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_items) {
        const Item it = items[i];
        out[i] = walk_start_of(plans[it.pad].g, it);
    }
}

template <bool DLP, int... Ps>
__device__ __forceinline__ void run_item_fp64(int p, const DevGeom &g, const DevEval &ev, const Item &it,
                                              const WalkStart &ws, double *T, int lane,
                                              std::integer_sequence<int, Ps...>)
{
    ((p == Ps ? (laplace_fp64_item<Ps, DLP, false>(g, ev, it, ws, T, kTile, lane), 0) : 0), ...);
}

template <bool DLP, int... Ps>
__device__ __forceinline__ void run_item_mixed(int p, const DevGeom &g, const DevEval &ev, const Item &it,
                                               const WalkStart &ws, float4 *T, int lane,
                                               std::integer_sequence<int, Ps...>)
{
    ((p == Ps ? (laplace_mixed_item<Ps, DLP, false>(g, ev, it, ws, T, kTile, lane), 0) : 0), ...);
}

template <int W, int... Ps>
__device__ __forceinline__ void run_part_item_mixed(int p, const DevGeom &g, const DevEval &ev, const Item &it,
                                                    const WalkStart &ws, int sl, std::integer_sequence<int, Ps...>)
{
    ((p == Ps ? (laplace_mixed_part_item<Ps, W>(g, ev, it, ws, sl), 0) : 0), ...);
}

template <int... Ps>
__device__ __forceinline__ void run_window4_mixed(int p, const DevGeom &g, const DevEval &ev, const Item &it,
                                                  int32_t a, int32_t b, int32_t A, int32_t B, float4 *T, int lane,
                                                  std::integer_sequence<int, Ps...>)
{
    ((p == Ps ? (laplace_mixed_window4<Ps>(g, ev, it, a, b, A, B, T, lane), 0) : 0), ...);
}

template <bool MIXED, bool DLP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, DLP ? 1 : 7)
batch_laplace_kernel(const BatchPlan *plans, const BatchIO *io, const Item *items, const WalkStart *walks,
                     int64_t n_items, unsigned long long *head)
{
    // per-warp tile at the default depth kTile (a batch stages every plan's
    // sources alike): mixed, pair records (laplace_items.cuh); FP64, one row per field
    constexpr int kWarpBytes = MIXED ? mixed_tile_rows(DLP) * (kTile / 2) * 16 : (DLP ? 7 : 4) * kTile * 8;
    __shared__ __align__(16) unsigned char tile_raw[kWarpsPerBlock * kWarpBytes];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        // pop kPopChunk consecutive items (similar cost: the queue is sorted)
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(head, (unsigned long long)kPopChunk);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (first >= (unsigned long long)n_items) break;       // queue drained
        const unsigned long long last = min(first + kPopChunk, (unsigned long long)n_items);
        for (unsigned long long idx = first; idx < last; ++idx) {
            const Item it = items[idx];
            const WalkStart ws = walks[idx];
            const BatchPlan &bp = plans[it.pad];
            DevEval ev = bp.ev;
            ev.out_slp = io[it.pad].out_slp;
            ev.out_dlp = io[it.pad].out_dlp;
            if constexpr (MIXED && !DLP) {
                // up to four single-target items of one plan: 8 or 16 lanes each
                int m = 0;
                if (it.n_tgt == 1)
                    for (m = 1; m < 4 && idx + m < last; ++m) {
                        const Item o = items[idx + m];
                        if (o.n_tgt != 1 || o.pad != it.pad) break;
                    }
                if (m >= 4) {
                    // four items whose lists are single runs with a short union:
                    // stage the union once for all four (item q = lane % 4, so
                    // that the lanes of the four items that read one staged
                    // record sit in one quarter-warp)
                    const int q = lane & 3;
                    const Item mine_it = items[idx + q];
                    int32_t a = 0, b = 0;
                    const bool run = single_run_range(mine_it, walks[idx + q], a, b);
                    const bool all_runs = __all_sync(0xffffffffu, run);
                    int32_t A = a, B = b, len = b - a;
#pragma unroll
                    for (int off = 1; off < 4; off <<= 1) {
                        A = min(A, __shfl_xor_sync(0xffffffffu, A, off));
                        B = max(B, __shfl_xor_sync(0xffffffffu, B, off));
                        len = max(len, __shfl_xor_sync(0xffffffffu, len, off));
                    }
                    if (all_runs && B - A <= 2 * len) {
                        run_window4_mixed(bp.p, bp.g, ev, mine_it, a, b, A, B,
                                          reinterpret_cast<float4 *>(tile_raw + warp * kWarpBytes), lane,
                                          std::make_integer_sequence<int, TSQBX_P_MAX + 1>{});
                        __syncwarp();
                        idx += 3;
                        continue;
                    }
                }
                if (m >= 2) {
                    const int W = m >= 4 ? 8 : 16;
                    const int q = lane / W;
                    const Item mine_it = items[idx + q];
                    const WalkStart mine_ws = walks[idx + q];
                    if (W == 8)
                        run_part_item_mixed<8>(bp.p, bp.g, ev, mine_it, mine_ws, lane & 7,
                                               std::make_integer_sequence<int, TSQBX_P_MAX + 1>{});
                    else
                        run_part_item_mixed<16>(bp.p, bp.g, ev, mine_it, mine_ws, lane & 15,
                                                std::make_integer_sequence<int, TSQBX_P_MAX + 1>{});
                    __syncwarp();
                    idx += 32 / W - 1;
                    continue;
                }
            }
            unsigned char *mine = tile_raw + warp * kWarpBytes;
            if constexpr (MIXED)
                run_item_mixed<DLP>(bp.p, bp.g, ev, it, ws, reinterpret_cast<float4 *>(mine), lane,
                                    std::make_integer_sequence<int, TSQBX_P_MAX + 1>{});
            else
                run_item_fp64<DLP>(bp.p, bp.g, ev, it, ws, reinterpret_cast<double *>(mine), lane,
                                   std::make_integer_sequence<int, TSQBX_P_MAX + 1>{});
            __syncwarp();
        }
    }
}

__global__ void batch_combine_kernel(const BatchPlan *plans, const BatchIO *io, const BatchCombine *rec,
                                     int64_t n_rec)
{
    const int64_t n = n_rec * 32;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const BatchCombine r = rec[i >> 5];
        const int j = (int)(i & 31);
        if (j >= r.c.n_tgt) continue;
        const BatchPlan &bp = plans[r.plan];
        const int64_t t = bp.g.slot_tgt[r.c.slot_begin + j];
        double a = 0.0, b = 0.0;
        for (int k = 0; k < r.c.n_slices; ++k) {
            const int64_t idx = (int64_t)r.c.part + (int64_t)k * r.c.n_tgt + j;
            if (bp.ev.part_slp) a += bp.ev.part_slp[idx];
            if (bp.ev.part_dlp) b += bp.ev.part_dlp[idx];
        }
        if (io[r.plan].out_slp) io[r.plan].out_slp[t] = a;
        if (io[r.plan].out_dlp) io[r.plan].out_dlp[t] = b;
    }
}

}  // namespace

struct tsqbx_batch_s {
    int device = 0;
    bool mixed = false, dlp = false, use_graph = true;
    int n_plans = 0;
    int64_t n_items = 0, n_combine = 0, max_src = 0;
    std::vector<tsqbx_plan> plans;
    std::vector<void *> dev;               // device allocations
    size_t device_bytes = 0;
    BatchPlan *d_plans = nullptr;
    BatchIO *d_io = nullptr;
    BatchIO *h_io = nullptr;               // pinned
    Item *d_items = nullptr;
    WalkStart *d_walks = nullptr;
    BatchCombine *d_combine = nullptr;
    unsigned long long *d_head = nullptr;
    int *d_status = nullptr;
    int grid = 0;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t io_done = nullptr, k_begin = nullptr, k_end = nullptr;
    bool launched = false;
    int64_t n_pairs = 0, n_pair_terms = 0;

    template <class T>
    T *dalloc(size_t count)
    {
        void *p = nullptr;
        ck(cudaMalloc(&p, (count ? count : 1) * sizeof(T)));
        dev.push_back(p);
        device_bytes += (count ? count : 1) * sizeof(T);
        return static_cast<T *>(p);
    }
    ~tsqbx_batch_s()
    {
        if (capture) cudaStreamSynchronize(capture);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (capture) cudaStreamDestroy(capture);
        for (cudaEvent_t e : {io_done, k_begin, k_end})
            if (e) cudaEventDestroy(e);
        if (h_io) cudaFreeHost(h_io);
        for (void *p : dev) cudaFree(p);
    }
};

namespace {

// The launch sequence of one batched evaluation (captured or issued directly).
// Events in the sequence are recorded with cudaEventRecordExternal while the
// sequence is being captured, so that graph replays record them.
cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing)
{
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

int issue(tsqbx_batch B, cudaStream_t s, bool capturing)
{
    ck(cudaMemcpyAsync(B->d_io, B->h_io, sizeof(BatchIO) * B->n_plans, cudaMemcpyHostToDevice, s));
    ck(record(B->io_done, s, capturing));
    if (B->max_src > 0) {
        dim3 grid((unsigned)std::min<int64_t>((B->max_src + 255) / 256, 64), (unsigned)B->n_plans);
        batch_prep_kernel<<<grid, 256, 0, s>>>(B->d_plans, B->d_io, B->mixed ? 1 : 0);
        ck(cudaGetLastError());
    }
    ck(cudaMemsetAsync(B->d_head, 0, sizeof(unsigned long long), s));
    ck(record(B->k_begin, s, capturing));
    if (B->n_items > 0) {
        const unsigned g = (unsigned)B->grid;
        if (B->mixed) {
            if (B->dlp) batch_laplace_kernel<true, true><<<g, kWarpsPerBlock * 32, 0, s>>>(B->d_plans, B->d_io, B->d_items, B->d_walks, B->n_items, B->d_head);
            else batch_laplace_kernel<true, false><<<g, kWarpsPerBlock * 32, 0, s>>>(B->d_plans, B->d_io, B->d_items, B->d_walks, B->n_items, B->d_head);
        } else {
            if (B->dlp) batch_laplace_kernel<false, true><<<g, kWarpsPerBlock * 32, 0, s>>>(B->d_plans, B->d_io, B->d_items, B->d_walks, B->n_items, B->d_head);
            else batch_laplace_kernel<false, false><<<g, kWarpsPerBlock * 32, 0, s>>>(B->d_plans, B->d_io, B->d_items, B->d_walks, B->n_items, B->d_head);
        }
        ck(cudaGetLastError());
    }
    if (B->n_combine > 0) {
        const int cb = (int)std::min<int64_t>((B->n_combine * 32 + 255) / 256, 2048);
        batch_combine_kernel<<<cb, 256, 0, s>>>(B->d_plans, B->d_io, B->d_combine, B->n_combine);
        ck(cudaGetLastError());
    }
    ck(record(B->k_end, s, capturing));
    return TSQBX_OK;
}

template <bool MIXED, bool DLP>
int occupancy(int *blocks)
{
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_laplace_kernel<MIXED, DLP>,
                                                              kWarpsPerBlock * 32, 0);
}

}  // namespace

extern "C" {

int tsqbx_batch_create(const tsqbx_plan *plans, int n_plans, int use_graph, tsqbx_batch *out)
{
    if (!out || !plans || n_plans < 1 || n_plans > 65535) return TSQBX_E_INVAL;
    *out = nullptr;
    const tsqbx_options &o0 = plans[0] ? plans[0]->opt : tsqbx_options{};
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return TSQBX_E_INVAL;
        const tsqbx_options &o = plans[i]->opt;
        if (o.kernel != TSQBX_LAPLACE || o.precision == TSQBX_DF64) return TSQBX_E_UNSUPPORTED;
        if (o.device != o0.device || o.precision != o0.precision || o.layers != o0.layers)
            return TSQBX_E_INVAL;
    }
    tsqbx_batch B = nullptr;
    try {
        DeviceGuard dg(o0.device);
        B = new tsqbx_batch_s;
        B->device = o0.device;
        B->mixed = o0.precision == TSQBX_MIXED;
        B->dlp = (o0.layers & TSQBX_DLP) != 0;
        B->use_graph = use_graph != 0;
        B->n_plans = n_plans;
        B->plans.assign(plans, plans + n_plans);
        // per-plan descriptors with batch-owned scratch
        std::vector<BatchPlan> bp(n_plans);
        struct Entry { Item it; double cost; };
        std::vector<Entry> items;
        std::vector<BatchCombine> comb;
        int n_sm = 152;
        for (int i = 0; i < n_plans; ++i) {
            tsqbx_plan P = plans[i];
            n_sm = P->n_sm;
            bp[i].g = P->g;
            bp[i].p = P->opt.p;
            DevEval &ev = bp[i].ev;
            const int64_t ns = P->g.n_src;
            B->max_src = std::max(B->max_src, ns);
            if (B->mixed) ev.wmu_f = B->dalloc<float>(ns);
            else ev.wmu = B->dalloc<double>(ns);
            const int64_t np = P->sched.n_parts;
            if (np && (P->opt.layers & TSQBX_SLP)) ev.part_slp = B->dalloc<double>(np);
            if (np && (P->opt.layers & TSQBX_DLP)) ev.part_dlp = B->dalloc<double>(np);
            for (const Schedule::Entry &e : P->sched.items) {
                Item it = e.it;
                it.pad = i;
                items.push_back({it, e.cost});
            }
            for (const Combine &c : P->sched.combine) comb.push_back({c, i});
            B->n_pairs += P->stats.n_pairs;
            B->n_pair_terms += P->stats.n_pair_terms;
        }
        B->d_status = B->dalloc<int>(1);
        ck(cudaMemset(B->d_status, 0, sizeof(int)));
        for (auto &p : bp) p.ev.status = B->d_status;
        std::vector<int32_t> plan_of(items.size());
        std::vector<double> cost(items.size());
        for (size_t k = 0; k < items.size(); ++k) {
            plan_of[k] = items[k].it.pad;
            cost[k] = items[k].cost;
        }
        const std::vector<int64_t> order = batch_queue_order(plan_of, cost);
        std::vector<Item> item_v(items.size());
        for (size_t k = 0; k < items.size(); ++k) item_v[k] = items[(size_t)order[k]].it;
        B->n_items = (int64_t)item_v.size();
        B->n_combine = (int64_t)comb.size();
        B->d_plans = B->dalloc<BatchPlan>(n_plans);
        ck(cudaMemcpy(B->d_plans, bp.data(), sizeof(BatchPlan) * n_plans, cudaMemcpyHostToDevice));
        B->d_items = B->dalloc<Item>(item_v.size());
        B->d_walks = B->dalloc<WalkStart>(item_v.size());
        if (!item_v.empty()) {
            ck(cudaMemcpy(B->d_items, item_v.data(), sizeof(Item) * item_v.size(), cudaMemcpyHostToDevice));
            const int64_t wb = ((int64_t)item_v.size() + 255) / 256;
            batch_walk_kernel<<<(unsigned)wb, 256>>>(B->d_plans, B->d_items, B->n_items, B->d_walks);
            ck(cudaGetLastError());
            ck(cudaStreamSynchronize(0));
        }
        B->d_combine = B->dalloc<BatchCombine>(comb.size());
        if (!comb.empty())
            ck(cudaMemcpy(B->d_combine, comb.data(), sizeof(BatchCombine) * comb.size(), cudaMemcpyHostToDevice));
        B->d_io = B->dalloc<BatchIO>(n_plans);
        B->d_head = B->dalloc<unsigned long long>(1);
        ck(cudaMallocHost(&B->h_io, sizeof(BatchIO) * n_plans));
        std::memset(B->h_io, 0, sizeof(BatchIO) * n_plans);
        ck(cudaEventCreateWithFlags(&B->io_done, cudaEventDisableTiming));
        ck(cudaEventCreate(&B->k_begin));
        ck(cudaEventCreate(&B->k_end));
        // persistent grid: one full wave of resident CTAs
        int per_sm = 1;
        ck(B->mixed ? (B->dlp ? (cudaError_t)occupancy<true, true>(&per_sm) : (cudaError_t)occupancy<true, false>(&per_sm))
                    : (B->dlp ? (cudaError_t)occupancy<false, true>(&per_sm) : (cudaError_t)occupancy<false, false>(&per_sm)));
        B->grid = std::max(1, per_sm) * n_sm;
        ck(cudaStreamCreateWithFlags(&B->capture, cudaStreamNonBlocking));
        if (B->use_graph) {
            ck(cudaStreamBeginCapture(B->capture, cudaStreamCaptureModeThreadLocal));
            int rc = TSQBX_OK;
            try {
                rc = issue(B, B->capture, true);
            } catch (const CudaFail &) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(B->capture, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            ck(cudaStreamEndCapture(B->capture, &B->graph));
            if (rc) { delete B; return rc; }
            ck(cudaGraphInstantiate(&B->exec, B->graph, 0));
        }
        *out = B;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        delete B;
        return status_of(f.err);
    } catch (const std::bad_alloc &) {
        delete B;
        return TSQBX_E_NOMEM;
    }
}

void tsqbx_batch_destroy(tsqbx_batch B)
{
    if (!B) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(B->device);
    delete B;
    if (prev >= 0) cudaSetDevice(prev);
}

int tsqbx_batch_eval_async(tsqbx_batch B, const void *const *d_density, void *const *d_out_slp,
                           void *const *d_out_dlp, void *stream)
{
    if (!B || !d_density) return TSQBX_E_INVAL;
    for (int i = 0; i < B->n_plans; ++i) {
        tsqbx_plan P = B->plans[i];
        if (P->g.n_src && !d_density[i]) return TSQBX_E_INVAL;
        if ((P->opt.layers & TSQBX_SLP) && P->g.n_tgt && (!d_out_slp || !d_out_slp[i])) return TSQBX_E_INVAL;
        if ((P->opt.layers & TSQBX_DLP) && P->g.n_tgt && (!d_out_dlp || !d_out_dlp[i])) return TSQBX_E_INVAL;
    }
    try {
        DeviceGuard dg(B->device);
        cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : B->capture;
        // the previous evaluation must have copied the pointer table first
        if (B->launched) ck(cudaEventSynchronize(B->io_done));
        for (int i = 0; i < B->n_plans; ++i) {
            B->h_io[i].density = static_cast<const double *>(d_density[i]);
            B->h_io[i].out_slp = d_out_slp ? static_cast<double *>(d_out_slp[i]) : nullptr;
            B->h_io[i].out_dlp = d_out_dlp ? static_cast<double *>(d_out_dlp[i]) : nullptr;
        }
        if (B->use_graph) ck(cudaGraphLaunch(B->exec, s));
        else {
            int rc = issue(B, s, false);
            if (rc) return rc;
        }
        B->launched = true;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    }
}

int tsqbx_batch_kernel_ms(tsqbx_batch B, float *ms)
{
    if (!B || !ms || !B->launched) return TSQBX_E_INVAL;
    try {
        DeviceGuard dg(B->device);
        ck(cudaEventSynchronize(B->k_end));
        ck(cudaEventElapsedTime(ms, B->k_begin, B->k_end));
        int st = 0;
        ck(cudaMemcpy(&st, B->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        return st ? TSQBX_E_KERNEL : TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    }
}

int tsqbx_batch_info(tsqbx_batch B, tsqbx_batch_stats *st)
{
    if (!B || !st) return TSQBX_E_INVAL;
    st->n_plans = B->n_plans;
    st->n_items = B->n_items;
    st->n_sliced = B->n_combine;
    st->n_pairs = B->n_pairs;
    st->n_pair_terms = B->n_pair_terms;
    st->grid_blocks = B->grid;
    st->graph = B->use_graph ? 1 : 0;
    st->launches_per_eval = (B->max_src > 0 ? 1 : 0) + (B->n_items > 0 ? 1 : 0) + (B->n_combine > 0 ? 1 : 0);
    st->device_bytes = B->device_bytes;
    return TSQBX_OK;
}

}  // extern "C"
