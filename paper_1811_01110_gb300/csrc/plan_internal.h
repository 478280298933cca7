// plan_internal.h -- host-side plan structures shared by plan.cu (plans,
// evaluation, tickets, tuning) and batch.cu (persistent batched launches).
#pragma once

#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "tsqbx.h"

namespace tsqbx {

struct CudaFail {
    cudaError_t err;
};

inline void ck(cudaError_t e)
{
    if (e != cudaSuccess) throw CudaFail{e};
}

// Name of the last CUDA error a library call on this thread ran into.
void note_cuda_error(cudaError_t e);

inline int status_of(cudaError_t e)
{
    note_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? TSQBX_E_NOMEM : TSQBX_E_CUDA;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) ck(cudaSetDevice(dev));
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// One group's share of the work: its targets are the slots
// [slot_begin, slot_begin + nt) and it lists ns sources.
struct GroupWork {
    int64_t q, slot_begin, nt, ns;
};

// How the work is cut into warp items.
struct Schedule {
    struct Entry { Item it; double cost; };
    std::vector<Entry> items;          // sorted by cost, heaviest first
    std::vector<Combine> combine;
    int64_t n_parts = 0;
    int lanes_policy = 0;              // 0 = per-group choice, else forced L
    int64_t max_iters = 0;             // cap on lane iterations per item
    double lane_utilisation = 1.0;
};

// Half-octave bucket of an item's estimated cost (queue order key).
int cost_bucket(double cost);
// Lanes per target chosen for a group: the fewest items * (lane iterations +
// staging + setup), with staging costing `staging` per listed source per 32
// lanes.  Staging weighs more where the per-pair arithmetic is cheap (the
// mixed kernels: kStagingMixed) than where it is heavy (FP64, df64).
constexpr double kStagingDefault = 0.25, kStagingMixed = 0.5;
int choose_lanes(int64_t nt, int64_t ns, double staging = kStagingDefault);
// Sources per conventional coefficient-formation item.
constexpr int64_t kConvSlice = 1024;
// Cost model (the form of the paper's Table 2, with this GPU's constants):
// whether a center with nt targets and ns listed sources is cheaper on the
// conventional path than on the target-specific one.
bool conventional_cheaper(int64_t nt, int64_t ns, int p, unsigned layers, bool helmholtz);
int size_priority(int64_t n_pairs, const tsqbx_options &o);
// The arithmetic of size_priority for a device priority range [greatest, least]
// (numerically greatest <= least): the pairs times a per-pair cost relative to
// Laplace FP64, one level per decade above 1e5, clamped to the range.
int priority_for_work(int64_t n_pairs, int kernel, int precision, int least, int greatest);
// Queue order of a persistent batch over several plans (item i of plan
// plan_of[i] with estimated cost cost[i]): plan by plan, the plans with the
// most work first, each plan's items heaviest first.  Running one surface's
// items together keeps its sources in L2; interleaving all surfaces by cost
// alone swept every surface's sources through L2 in each cost bucket.
std::vector<int64_t> batch_queue_order(const std::vector<int32_t> &plan_of, const std::vector<double> &cost);
// Build the schedule; max_iters <= 0 picks the automatic cap; `staging` as
// in choose_lanes (used when lanes_policy is 0).
int build_schedule(const std::vector<GroupWork> &groups, int lanes_policy, int64_t max_iters,
                   int n_sm, Schedule &out, double staging = kStagingDefault);

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void *d_density = nullptr;     // device copy of a host density
    void *d_wmu = nullptr;         // w mu scratch (f64, f32 or c128)
    double *d_out[3] = {nullptr, nullptr, nullptr};    // single layer, double layer, S'
    double *d_part[3] = {nullptr, nullptr, nullptr};   // partial sums of sliced items
    int *d_status = nullptr;
    double *d_conv = nullptr;      // conventional partial coefficients
    void *h_density = nullptr;     // pinned staging
    void *h_out[3] = {nullptr, nullptr, nullptr};
    int *h_status = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    void *user_out[3] = {nullptr, nullptr, nullptr};
    bool copy_out[3] = {false, false, false};
    // outputs of a tsqbx_submit_multi / tsqbx_submit_multi_layers call:
    // layer l (0 single, 1 double) of density r
    int n_rhs = 1;
    void *user_out_rhs[2][kMaxRhs] = {};
    bool copy_out_rhs[2][kMaxRhs] = {};
};

}  // namespace tsqbx

struct tsqbx_plan_s {
    tsqbx_options opt{};
    tsqbx::DevGeom g;
    std::unordered_map<void *, size_t> dev_allocs;
    std::vector<void *> host_allocs;
    size_t device_bytes = 0;
    tsqbx_plan_stats stats{};
    std::vector<tsqbx::Slot> slots;
    std::mutex mu;
    size_t density_bytes = 0, out_bytes = 0, wmu_bytes = 0;
    size_t conv_coef_doubles = 0;                     // per slot, for the plan's p
    cudaEvent_t k_begin = nullptr, k_end = nullptr;   // brackets the expansion (slot 0)
    bool k_timed = false;
    int n_sm = 152;
    std::vector<tsqbx::GroupWork> groups;             // kept for rescheduling
    tsqbx::Schedule sched;                            // host copy of the current items
    std::vector<double> list_hist;                    // tuning-cache signature

    template <class T>
    T *dalloc(size_t count)
    {
        if (count == 0) count = 1;
        void *p = nullptr;
        tsqbx::ck(cudaMalloc(&p, count * sizeof(T)));
        dev_allocs[p] = count * sizeof(T);
        device_bytes += count * sizeof(T);
        return static_cast<T *>(p);
    }
    void dfree(const void *cp)
    {
        void *p = const_cast<void *>(cp);
        auto it = dev_allocs.find(p);
        if (it == dev_allocs.end()) return;
        device_bytes -= it->second;
        dev_allocs.erase(it);
        cudaFree(p);
    }
    template <class T>
    T *upload(const std::vector<T> &v)
    {
        T *p = dalloc<T>(v.size());
        if (!v.empty()) tsqbx::ck(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return p;
    }
    void *halloc(size_t bytes)
    {
        void *p = nullptr;
        tsqbx::ck(cudaMallocHost(&p, bytes ? bytes : 1));
        host_allocs.push_back(p);
        return p;
    }
    ~tsqbx_plan_s();
};

namespace tsqbx {

// Install a schedule on a plan: upload items and combine records, size the
// partial-sum buffers of every slot (frees what the old schedule used).
void apply_schedule(tsqbx_plan P, Schedule &&s);
// Densities a slot's buffers hold: o.max_rhs (0 = 1).
inline int rhs_capacity(const tsqbx_options &o) { return o.max_rhs > 1 ? o.max_rhs : 1; }
// Enqueue prep + expansion (+ combine) for one evaluation on stream s, with
// expansion order p and (Helmholtz) wavenumber k; S' is formed only when the
// plan's mask has it and d_sp is given.
int enqueue(tsqbx_plan P, Slot &slot, const void *d_density, double *d_slp, double *d_dlp, double *d_sp,
            cudaStream_t s, bool timed, int p, double k);

}  // namespace tsqbx
