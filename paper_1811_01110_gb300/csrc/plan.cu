// plan.cu -- host side of libtsqbx: plan construction (validation, grouping of
// targets, work schedule, packing and upload of source/target records, the
// convergence check), evaluation, submit/poll tickets and the autotuner.
//
// The C ABI is declared in include/tsqbx.h; every entry point below traps C++
// exceptions and converts CUDA failures into TSQBX_E_* codes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "plan_internal.h"

using namespace tsqbx;

static_assert(kPMax == TSQBX_P_MAX, "the kernels' coefficient tables cover every order");

namespace {

// ------------------------------------------------------------- prep kernels

// Per-evaluation source weights times density, w_s mu_s, in the form each
// kernel family stages.
__global__ void prep_wmu_fp64(const double4_32a *src_pw, const double *mu, int64_t n, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src_pw[i].w * mu[i];
}

__global__ void prep_wmu_f32(const double4_32a *src_pw, const double *mu, int64_t n, float *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(src_pw[i].w * mu[i]);
}

__global__ void prep_wmu_c128(const double4_32a *src_pw, const double2 *mu, int64_t n, double2 *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double w = src_pw[i].w;
        const double2 m = mu[i];
        out[i] = make_double2(w * m.x, w * m.y);
    }
}

// Convergence check over every listed pair (same item walk as the kernels):
// Where each item's slice starts in its group's run list (WalkStart).
__global__ void walk_start_kernel(const DevGeom g, WalkStart *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.n_items) out[i] = walk_start_of(g, g.items[i]);
}

// counts |t-c|^2 >= |s-c|^2 (outside the expansion's region of convergence,
// Appendix A) and s == c.
__global__ void check_pairs_kernel(const DevGeom g, unsigned long long *n_div,
                                   unsigned long long *n_zero)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    const Item it = g.items[item];
    unsigned long long nd = 0, nz = 0;
    for (int j = 0; j < it.n_tgt; ++j) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double rho2 = g.slot_e[it.slot_begin + j].w;
        ListWalk walk(g, it.group);
        for (int k = it.src_lo + lane; k < it.src_hi; k += 32) {
            const int s = walk.at(k);
            if ((unsigned)s >= (unsigned)g.n_src) continue;
            const double4_32a p = g.src_pw[s];
            const double dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
            const double R2 = dx * dx + dy * dy + dz * dz;
            if (R2 == 0.0) ++nz;
            else if (rho2 >= R2) ++nd;
        }
    }
    if (nd) atomicAdd(n_div, nd);
    if (nz) atomicAdd(n_zero, nz);
}

// Second pass for sliced items: each target's partial sums (one per slice of
// its group's list) are added in slice order, so results are deterministic.
__global__ void combine_kernel(const DevGeom g, const double *part_slp, const double *part_dlp,
                               const double *part_sp, double *out_slp, double *out_dlp, double *out_sp,
                               int width)
{
    const int64_t n = g.n_combine * 32;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Combine r = g.combine[i >> 5];
        const int j = (int)(i & 31);
        if (j >= r.n_tgt) continue;
        const int64_t t = g.slot_tgt[r.slot_begin + j];
        for (int w = 0; w < width; ++w) {
            double a = 0.0, b = 0.0, c = 0.0;
            for (int k = 0; k < r.n_slices; ++k) {
                const int64_t idx = ((int64_t)r.part + (int64_t)k * r.n_tgt + j) * width + w;
                if (part_slp) a += part_slp[idx];
                if (part_dlp) b += part_dlp[idx];
                if (part_sp) c += part_sp[idx];
            }
            if (out_slp) out_slp[t * width + w] = a;
            if (out_dlp) out_dlp[t * width + w] = b;
            if (out_sp) out_sp[t * width + w] = c;
        }
    }
}

// ------------------------------------------------------------------ helpers

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline bool finite3(const double *xyz, int64_t n, int64_t i)
{
    return std::isfinite(xyz[i]) && std::isfinite(xyz[n + i]) && std::isfinite(xyz[2 * n + i]);
}

void split_ff(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

std::mutex g_ticket_mu;
std::unordered_map<uint64_t, std::pair<tsqbx_plan, int>> g_tickets;
std::atomic<uint64_t> g_next_ticket{1};

// Process-wide tuning cache: (kernel, precision, p, layers, list shape) -> tuning.
using TuneKey = std::tuple<int, int, int, unsigned, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, tsqbx_tuning> g_tune_cache;

TuneKey tune_key(tsqbx_plan P)
{
    // list shape: half-octave buckets of the mean sources per group and the
    // mean targets per group (what the lane choice and slicing depend on)
    const double ns = P->list_hist.size() > 0 ? P->list_hist[0] : 0.0;
    const double nt = P->list_hist.size() > 1 ? P->list_hist[1] : 0.0;
    const int bs = ns > 0 ? (int)std::lround(2.0 * std::log2(ns)) : -1;
    const int bt = nt > 0 ? (int)std::lround(2.0 * std::log2(nt)) : -1;
    return TuneKey{(int)P->opt.kernel, (int)P->opt.precision, P->opt.p, P->opt.layers, bs, bt};
}

// The order-loop forms (tsqbx_options.p_unroll): 0 (per-order kernels) or the
// runtime-order kernel's unroll factor 1, 2 or 4; the latter exist for the
// Laplace FP64 and mixed kernels.
bool p_unroll_ok(int u) { return u == 0 || u == 1 || u == 2 || u == 4; }
bool has_runtime_order(int kernel, int precision)
{
    return kernel == TSQBX_LAPLACE && (precision == TSQBX_FP64 || precision == TSQBX_MIXED);
}
// Weight of source staging in the per-group lane choice: the mixed kernels'
// per-pair arithmetic is cheap, so their staging weighs more (measured on the
// torus: mixed 1.008 -> 0.994 ms at 0.5; df64 best at 0.25).
double staging_weight(const tsqbx_plan_s *P)
{
    return P->opt.precision == TSQBX_MIXED ? kStagingMixed : kStagingDefault;
}
// FP64 items inside the double-float launch (tsqbx_options.fp64_share).
bool has_both_pipes(int kernel, int precision) { return kernel == TSQBX_LAPLACE && precision == TSQBX_DF64; }
// Several densities per evaluation (tsqbx_options.max_rhs > 1,
// tsqbx_submit_multi_layers): the single layer of Helmholtz plans; the single
// and/or double layer (no S') of Laplace plans in FP64 or double-float.
bool multi_ok(const tsqbx_options &o)
{
    if (o.kernel == TSQBX_HELMHOLTZ) return o.layers == TSQBX_SLP;
    return o.kernel == TSQBX_LAPLACE && o.precision != TSQBX_MIXED && o.layers != 0 &&
           !(o.layers & ~(uint32_t)(TSQBX_SLP | TSQBX_DLP));
}

// Forget the per-density outputs of a multi-density call.
void reset_multi(Slot &slot)
{
    slot.n_rhs = 1;
    for (auto &l : slot.copy_out_rhs)
        for (bool &c : l) c = false;
}

int validate(const tsqbx_geometry *G, const tsqbx_options *o)
{
    if (!G || !o) return TSQBX_E_INVAL;
    if (o->kernel != TSQBX_LAPLACE && o->kernel != TSQBX_HELMHOLTZ) return TSQBX_E_INVAL;
    if (o->layers == 0 || (o->layers & ~(uint32_t)(TSQBX_SLP | TSQBX_DLP | TSQBX_SP))) return TSQBX_E_INVAL;
    if (o->p < 0 || o->p > TSQBX_P_MAX) return TSQBX_E_INVAL;
    if (o->precision != TSQBX_FP64 && o->precision != TSQBX_MIXED && o->precision != TSQBX_DF64)
        return TSQBX_E_INVAL;
    if (o->lanes_per_target < 0 || o->lanes_per_target > 32 || o->n_slots < 0 || o->n_slots > 64 ||
        o->max_item_iters < 0 || (o->tile_depth != 0 && !tsqbx::tile_depth_ok(o->tile_depth)) ||
        o->max_rhs < 0 || o->max_rhs > tsqbx::kMaxRhs || !p_unroll_ok(o->p_unroll) ||
        o->fp64_share < 0 || o->fp64_share > 20)
        return TSQBX_E_INVAL;
    if (o->kernel == TSQBX_HELMHOLTZ) {
        if (!(o->k > 0.0) || !std::isfinite(o->k)) return TSQBX_E_INVAL;
        if (o->precision != TSQBX_FP64) return TSQBX_E_UNSUPPORTED;
    }
    if ((o->flags & (TSQBX_FLAG_CONVENTIONAL_AUTO | TSQBX_FLAG_CONVENTIONAL_ALL)) && o->precision != TSQBX_FP64)
        return TSQBX_E_UNSUPPORTED;
    if ((o->flags & TSQBX_FLAG_CONVENTIONAL_ALL) && o->kernel == TSQBX_HELMHOLTZ && o->p > kConvHelmMaxP)
        return TSQBX_E_UNSUPPORTED;
    // several densities per evaluation: the single layer, Helmholtz or Laplace
    // in FP64 or double-float
    if (o->max_rhs > 1 && !multi_ok(*o)) return TSQBX_E_UNSUPPORTED;
    // runtime-order kernels: Laplace FP64 and mixed only
    if (o->p_unroll != 0 && !has_runtime_order(o->kernel, o->precision)) return TSQBX_E_UNSUPPORTED;
    // FP64 items inside the double-float launch: Laplace df64 only
    if (o->fp64_share != 0 && !has_both_pipes(o->kernel, o->precision)) return TSQBX_E_UNSUPPORTED;
    if (G->n_src < 0 || G->n_ctr < 0 || G->n_tgt < 0 || G->n_group < 0) return TSQBX_E_INVAL;
    if (G->n_src > INT32_MAX || G->n_ctr > INT32_MAX || G->n_tgt > INT32_MAX || G->n_group > INT32_MAX)
        return TSQBX_E_INVAL;
    if ((G->n_src && (!G->src_xyz || !G->src_weight)) || (G->n_ctr && !G->ctr_xyz) ||
        (G->n_tgt && (!G->tgt_xyz || !G->tgt_center)) || (G->n_ctr && !G->ctr_group) ||
        !G->group_range_start)
        return TSQBX_E_INVAL;
    if ((o->layers & TSQBX_DLP) && G->n_src && !G->src_normal) return TSQBX_E_INVAL;
    if ((o->layers & TSQBX_SP) && G->n_tgt && !G->tgt_normal) return TSQBX_E_INVAL;
    if (G->group_range_start[0] != 0) return TSQBX_E_INVAL;
    for (int64_t q = 0; q < G->n_group; ++q)
        if (G->group_range_start[q + 1] < G->group_range_start[q]) return TSQBX_E_INVAL;
    const int64_t nnz = G->group_range_start[G->n_group];
    if (nnz > 0 && (!G->range_begin || !G->range_end)) return TSQBX_E_INVAL;
    for (int64_t i = 0; i < nnz; ++i)
        if (G->range_begin[i] < 0 || G->range_end[i] < G->range_begin[i] ||
            G->range_end[i] > G->n_src)
            return TSQBX_E_INVAL;
    for (int64_t t = 0; t < G->n_tgt; ++t) {
        if (G->tgt_center[t] < 0 || G->tgt_center[t] >= G->n_ctr || !finite3(G->tgt_xyz, G->n_tgt, t))
            return TSQBX_E_INVAL;
        if ((o->layers & TSQBX_SP) && !finite3(G->tgt_normal, G->n_tgt, t)) return TSQBX_E_INVAL;
    }
    for (int64_t c = 0; c < G->n_ctr; ++c)
        if (G->ctr_group[c] < 0 || G->ctr_group[c] >= G->n_group || !finite3(G->ctr_xyz, G->n_ctr, c))
            return TSQBX_E_INVAL;
    for (int64_t s = 0; s < G->n_src; ++s) {
        if (!finite3(G->src_xyz, G->n_src, s) || !std::isfinite(G->src_weight[s])) return TSQBX_E_INVAL;
        if ((o->layers & TSQBX_DLP) && !finite3(G->src_normal, G->n_src, s)) return TSQBX_E_INVAL;
    }
    return TSQBX_OK;
}

void fill_stats(tsqbx_plan P)
{
    tsqbx_plan_stats &st = P->stats;
    st.n_items = P->g.n_items;
    st.lane_utilisation = P->sched.lane_utilisation;
    st.device_bytes = P->device_bytes;
    st.n_sliced = (int64_t)P->sched.combine.size();
    st.launches_per_eval = (P->g.n_src > 0 ? 1 : 0) + (P->g.n_items > 0 ? 1 : 0) + (st.n_sliced > 0 ? 1 : 0) +
                           (P->g.n_conv_items > 0 ? 1 : 0) + (P->g.n_conv_eval > 0 ? 1 : 0);
}

}  // namespace

// ---------------------------- errors, stream priority, schedule upload
// (the schedule itself is built in schedule.cu)

namespace tsqbx {

static thread_local const char *t_last_error = "no error";

void note_cuda_error(cudaError_t e) { t_last_error = cudaGetErrorName(e); }

// Stream priority of a plan under TSQBX_FLAG_SIZE_PRIORITY: one level per
// decade of work (pairs times a cost per pair relative to Laplace FP64) above
// 1e5, from the device's highest priority for the smallest plans down to its
// lowest.
int size_priority(int64_t n_pairs, const tsqbx_options &o)
{
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return priority_for_work(n_pairs, o.kernel, o.precision, least, greatest);
}

void apply_schedule(tsqbx_plan P, Schedule &&s)
{
    const bool helm = P->opt.kernel == TSQBX_HELMHOLTZ;
    std::vector<Item> items(s.items.size());
    for (size_t i = 0; i < items.size(); ++i) items[i] = s.items[i].it;
    if (P->g.items) P->dfree(P->g.items);
    if (P->g.combine) P->dfree(P->g.combine);
    P->g.items = nullptr;
    P->g.combine = nullptr;
    for (Slot &sl : P->slots)
        for (int l = 0; l < 3; ++l) {
            if (sl.d_part[l]) P->dfree(sl.d_part[l]);
            sl.d_part[l] = nullptr;
        }
    P->g.items = P->upload(items);
    P->g.combine = P->upload(s.combine);
    P->g.n_items = (int64_t)items.size();
    if (P->g.item_walk) P->dfree(P->g.item_walk);
    WalkStart *walks = P->dalloc<WalkStart>(items.size());
    P->g.item_walk = walks;
    if (!items.empty()) {
        const int64_t blocks = ((int64_t)items.size() + 255) / 256;
        walk_start_kernel<<<(unsigned)blocks, 256>>>(P->g, walks);
        ck(cudaGetLastError());
        ck(cudaStreamSynchronize(0));
    }
    P->g.n_combine = (int64_t)s.combine.size();
    P->g.n_parts = s.n_parts;
    const size_t part_doubles = (size_t)s.n_parts * (helm ? 2 : 1);
    for (Slot &sl : P->slots) {
        if (s.n_parts && (P->opt.layers & TSQBX_SLP))
            sl.d_part[0] = P->dalloc<double>(part_doubles * (size_t)rhs_capacity(P->opt));
        if (s.n_parts && (P->opt.layers & TSQBX_DLP))
            sl.d_part[1] = P->dalloc<double>(part_doubles * (size_t)rhs_capacity(P->opt));
        if (s.n_parts && (P->opt.layers & TSQBX_SP)) sl.d_part[2] = P->dalloc<double>(part_doubles);
    }
    P->sched = std::move(s);
    fill_stats(P);
}

int enqueue(tsqbx_plan P, Slot &slot, const void *d_density, double *d_slp, double *d_dlp, double *d_sp,
            cudaStream_t s, bool timed, int p, double k)
{
    const tsqbx_options &o = P->opt;
    if (P->g.n_conv_centers > 0 && p > o.p) return TSQBX_E_UNSUPPORTED;   // coefficient scratch sized for o.p
    const int64_t n = P->g.n_src;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)P->n_sm * 16);
    DevEval ev;
    ev.status = slot.d_status;
    ev.out_slp = (o.layers & TSQBX_SLP) ? d_slp : nullptr;
    ev.out_dlp = (o.layers & TSQBX_DLP) ? d_dlp : nullptr;
    ev.out_sp = (o.layers & TSQBX_SP) ? d_sp : nullptr;
    ev.part_slp = slot.d_part[0];
    ev.part_dlp = slot.d_part[1];
    ev.part_sp = ev.out_sp ? slot.d_part[2] : nullptr;
    ev.k = k;
    ev.p = p;
    ev.conv_coef = slot.d_conv;
    if (n > 0) {
        if (o.kernel == TSQBX_HELMHOLTZ) {
            prep_wmu_c128<<<blocks, threads, 0, s>>>(P->g.src_pw, static_cast<const double2 *>(d_density), n,
                                                     static_cast<double2 *>(slot.d_wmu));
        } else if (o.precision == TSQBX_MIXED) {
            prep_wmu_f32<<<blocks, threads, 0, s>>>(P->g.src_pw, static_cast<const double *>(d_density), n,
                                                    static_cast<float *>(slot.d_wmu));
        } else {
            prep_wmu_fp64<<<blocks, threads, 0, s>>>(P->g.src_pw, static_cast<const double *>(d_density), n,
                                                     static_cast<double *>(slot.d_wmu));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return status_of(e);
    }
    ev.wmu = static_cast<const double *>(slot.d_wmu);
    ev.wmu_f = static_cast<const float *>(slot.d_wmu);
    ev.wmu_c = static_cast<const double2 *>(slot.d_wmu);
    // S' is formed only when the call asks for it (an S' output was given)
    const unsigned layers = ev.out_sp ? o.layers : (o.layers & ~(unsigned)TSQBX_SP);
    if (timed) ck(cudaEventRecord(P->k_begin, s));
    int rc;
    if (o.kernel == TSQBX_HELMHOLTZ) rc = launch_helmholtz_fp64(p, layers, P->g, ev, s);
    else if (o.precision == TSQBX_MIXED) rc = launch_laplace_mixed(p, layers, P->g, ev, s);
    else if (o.precision == TSQBX_DF64) rc = launch_laplace_df64(p, layers, P->g, ev, s);
    else rc = launch_laplace_fp64(p, layers, P->g, ev, s);
    if (rc != 0) return status_of((cudaError_t)rc);
    if (P->g.n_conv_centers > 0) {
        rc = o.kernel == TSQBX_HELMHOLTZ ? launch_conventional_helm(p, layers, P->g, ev, s)
                                         : launch_conventional(p, layers, P->g, ev, s);
        if (rc != 0) return status_of((cudaError_t)rc);
    }
    if (P->g.n_combine > 0) {
        const int64_t th = P->g.n_combine * 32;
        const int cb = (int)std::min<int64_t>((th + 255) / 256, (int64_t)P->n_sm * 8);
        combine_kernel<<<cb, 256, 0, s>>>(P->g, ev.part_slp, ev.part_dlp, ev.part_sp, ev.out_slp, ev.out_dlp,
                                          ev.out_sp, o.kernel == TSQBX_HELMHOLTZ ? 2 : 1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return status_of(e);
    }
    if (timed) {
        ck(cudaEventRecord(P->k_end, s));
        P->k_timed = true;
    }
    return TSQBX_OK;
}

// Enqueue one evaluation for n densities (the first at d_density, the others
// at steps of density_bytes, or the n pointers d_densities) of the plan's
// single layer into d_outs[0][r] and, for Laplace, its double layer into
// d_outs[1][r]: w mu of each density, the multi-density expansion kernel of
// the plan's kernel and precision, and the slice combine per density.
int enqueue_multi(tsqbx_plan P, Slot &slot, int n, const void *d_density, const void *const *d_densities,
                  double *const (&d_outs)[2][kMaxRhs], cudaStream_t s, int p, double k)
{
    const tsqbx_options &o = P->opt;
    const bool helm = o.kernel == TSQBX_HELMHOLTZ;
    const bool slp = (o.layers & TSQBX_SLP) != 0, dlp = !helm && (o.layers & TSQBX_DLP) != 0;
    const int64_t ns = P->g.n_src;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((ns + threads - 1) / threads, (int64_t)P->n_sm * 16);
    for (int r = 0; r < n && ns > 0; ++r) {
        const char *dens = d_densities ? static_cast<const char *>(d_densities[r])
                                       : static_cast<const char *>(d_density) + (size_t)r * P->density_bytes;
        if (helm)
            prep_wmu_c128<<<blocks, threads, 0, s>>>(P->g.src_pw, reinterpret_cast<const double2 *>(dens), ns,
                                                     static_cast<double2 *>(slot.d_wmu) + (size_t)r * ns);
        else
            prep_wmu_fp64<<<blocks, threads, 0, s>>>(P->g.src_pw, reinterpret_cast<const double *>(dens), ns,
                                                     static_cast<double *>(slot.d_wmu) + (size_t)r * ns);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return status_of(e);
    }
    DevEval ev;
    ev.status = slot.d_status;
    ev.out_slp = slp ? d_outs[0][0] : nullptr;
    ev.out_dlp = dlp ? d_outs[1][0] : nullptr;
    ev.part_slp = slp ? slot.d_part[0] : nullptr;
    ev.part_dlp = dlp ? slot.d_part[1] : nullptr;
    ev.k = k;
    ev.p = p;
    ev.wmu = static_cast<const double *>(slot.d_wmu);
    ev.wmu_c = static_cast<const double2 *>(slot.d_wmu);
    ev.n_rhs = n;
    ev.rhs_src_stride = ns;
    ev.rhs_part_stride = (helm ? 2 : 1) * P->g.n_parts;
    for (int r = 0; r < n; ++r) {
        ev.out_rhs[r] = slp ? d_outs[0][r] : nullptr;
        ev.out_rhs_dlp[r] = dlp ? d_outs[1][r] : nullptr;
    }
    const unsigned layers = (slp ? TSQBX_SLP : 0u) | (dlp ? TSQBX_DLP : 0u);
    int rc;
    if (helm)
        rc = n == 1 ? launch_helmholtz_fp64(p, TSQBX_SLP, P->g, ev, s) : launch_helmholtz_multi(p, P->g, ev, s);
    else if (o.precision == TSQBX_DF64)
        rc = n == 1 ? launch_laplace_df64(p, layers, P->g, ev, s) : launch_laplace_df64_multi(p, dlp, P->g, ev, s);
    else
        rc = n == 1 ? launch_laplace_fp64(p, layers, P->g, ev, s) : launch_laplace_fp64_multi(p, dlp, P->g, ev, s);
    if (rc != 0) return status_of((cudaError_t)rc);
    if (P->g.n_combine > 0) {
        const int64_t th = P->g.n_combine * 32;
        const int cb = (int)std::min<int64_t>((th + 255) / 256, (int64_t)P->n_sm * 8);
        for (int r = 0; r < n; ++r) {
            combine_kernel<<<cb, 256, 0, s>>>(P->g, ev.part_slp ? ev.part_slp + r * ev.rhs_part_stride : nullptr,
                                              ev.part_dlp ? ev.part_dlp + r * ev.rhs_part_stride : nullptr,
                                              nullptr, ev.out_rhs[r], ev.out_rhs_dlp[r], nullptr, helm ? 2 : 1);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return status_of(e);
        }
    }
    return TSQBX_OK;
}

}  // namespace tsqbx

tsqbx_plan_s::~tsqbx_plan_s()
{
    for (auto &s : slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (k_begin) cudaEventDestroy(k_begin);
    if (k_end) cudaEventDestroy(k_end);
    for (auto &kv : dev_allocs) cudaFree(kv.first);
    for (void *p : host_allocs) cudaFreeHost(p);
}

extern "C" {

int tsqbx_version(void) { return 10500; }

const char *tsqbx_last_error(void) { return t_last_error; }

const char *tsqbx_strerror(int status)
{
    switch (status) {
    case TSQBX_OK: return "ok";
    case TSQBX_PENDING: return "pending: work still in flight";
    case TSQBX_E_INVAL: return "invalid argument (size, pointer, index range or order)";
    case TSQBX_E_DIVERGENT: return "a listed pair has |t-c| >= |s-c| or s == c";
    case TSQBX_E_NOMEM: return "out of device or pinned host memory";
    case TSQBX_E_CUDA: return "CUDA runtime error";
    case TSQBX_E_TIMEOUT: return "timed out";
    case TSQBX_E_BUSY: return "every slot of the plan is in flight";
    case TSQBX_E_NOTFOUND: return "unknown or already collected ticket";
    case TSQBX_E_KERNEL: return "a kernel found an out-of-range source index";
    case TSQBX_E_UNSUPPORTED: return "kernel/layer/precision combination not provided";
    case TSQBX_E_TOO_LARGE: return "more sources than the fixed no-allocation scratch holds";
    default: return "unknown status";
    }
}

int tsqbx_plan_create(const tsqbx_geometry *G, const tsqbx_options *o, tsqbx_plan *out)
{
    if (!out) return TSQBX_E_INVAL;
    *out = nullptr;
    int rc = validate(G, o);
    if (rc) return rc;
    tsqbx_plan P = nullptr;
    try {
        DeviceGuard dg(o->device);
        P = new tsqbx_plan_s;
        P->opt = *o;
        if (P->opt.n_slots == 0) P->opt.n_slots = 2;
        {
            int v = 0;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, o->device) == cudaSuccess && v > 0)
                P->n_sm = v;
            cudaGetLastError();
        }
        const bool dlp = (o->layers & TSQBX_DLP) != 0;
        const bool sp = (o->layers & TSQBX_SP) != 0;
        const bool mixed = o->precision == TSQBX_MIXED;
        const int64_t n_src = G->n_src, n_tgt = G->n_tgt, n_group = G->n_group;

        // list length of each group (prefix sums)
        std::vector<int64_t> grp_off(n_group + 1, 0);
        for (int64_t q = 0; q < n_group; ++q) {
            int64_t ns = 0;
            for (int64_t r = G->group_range_start[q]; r < G->group_range_start[q + 1]; ++r)
                ns += G->range_end[r] - G->range_begin[r];
            if (ns > INT32_MAX) { delete P; return TSQBX_E_INVAL; }
            grp_off[q + 1] = grp_off[q] + ns;
        }
        // the lists as merged runs: a range that continues the previous one
        // extends its run; empty ranges add nothing
        std::vector<int32_t> grp_run(n_group + 1, 0), run_end, run_src;
        for (int64_t q = 0; q < n_group; ++q) {
            int32_t at = 0, prev_end = -1;
            for (int64_t r = G->group_range_start[q]; r < G->group_range_start[q + 1]; ++r) {
                const int32_t b = G->range_begin[r], e = G->range_end[r];
                if (e <= b) continue;
                at += e - b;
                if (b == prev_end) {
                    run_end.back() = at;
                } else {
                    run_end.push_back(at);
                    run_src.push_back(b);
                }
                prev_end = e;
            }
            if (run_end.size() > (size_t)INT32_MAX - 1) { delete P; return TSQBX_E_INVAL; }
            grp_run[q + 1] = (int32_t)run_end.size();
        }
        // path of each center: conventional QBX or target-specific
        const int64_t n_ctr = G->n_ctr;
        std::vector<int64_t> ctr_nt(n_ctr, 0);
        for (int64_t t = 0; t < n_tgt; ++t) ++ctr_nt[G->tgt_center[t]];
        std::vector<char> conv(n_ctr, 0);
        const bool conv_ok = o->kernel != TSQBX_HELMHOLTZ || o->p <= kConvHelmMaxP;
        if ((o->flags & (TSQBX_FLAG_CONVENTIONAL_AUTO | TSQBX_FLAG_CONVENTIONAL_ALL)) && conv_ok) {
            const bool all = (o->flags & TSQBX_FLAG_CONVENTIONAL_ALL) != 0;
            for (int64_t c = 0; c < n_ctr; ++c) {
                if (ctr_nt[c] == 0) continue;
                const int64_t q = G->ctr_group[c];
                conv[c] = all || conventional_cheaper(ctr_nt[c], grp_off[q + 1] - grp_off[q], o->p, o->layers,
                                                      o->kernel == TSQBX_HELMHOLTZ);
            }
        }
        // target slots: by group; within a group the target-specific targets
        // first (input order), then each conventional center's targets
        // (center order, then input order), contiguous per center
        std::vector<int64_t> tcount(n_group + 1, 0), ts_count(n_group, 0);
        for (int64_t t = 0; t < n_tgt; ++t) {
            const int64_t c = G->tgt_center[t], q = G->ctr_group[c];
            ++tcount[q + 1];
            if (!conv[c]) ++ts_count[q];
        }
        for (int64_t q = 0; q < n_group; ++q) tcount[q + 1] += tcount[q];
        std::vector<int32_t> slot_tgt(n_tgt);
        std::vector<ConvCenter> conv_centers;
        std::vector<int64_t> conv_pos(n_ctr, -1);
        {
            std::vector<int64_t> pos_ts(tcount.begin(), tcount.end() - 1), pos_cv(n_group);
            for (int64_t q = 0; q < n_group; ++q) pos_cv[q] = tcount[q] + ts_count[q];
            for (int64_t c = 0; c < n_ctr; ++c) {
                if (!conv[c]) continue;
                const int64_t q = G->ctr_group[c];
                conv_pos[c] = pos_cv[q];
                conv_centers.push_back(ConvCenter{(int32_t)q, (int32_t)pos_cv[q], (int32_t)ctr_nt[c], 0, 0, 0, 0, 0});
                pos_cv[q] += ctr_nt[c];
            }
            for (int64_t t = 0; t < n_tgt; ++t) {
                const int64_t c = G->tgt_center[t];
                if (conv[c]) slot_tgt[conv_pos[c]++] = (int32_t)t;
                else slot_tgt[pos_ts[G->ctr_group[c]]++] = (int32_t)t;
            }
        }
        int64_t n_pairs = 0, n_busy = 0;
        double sum_ns = 0.0;
        std::vector<GroupWork> all_groups;              // every target (convergence check)
        for (int64_t q = 0; q < n_group; ++q) {
            const int64_t nt = tcount[q + 1] - tcount[q];
            if (nt == 0) continue;
            const int64_t ns = grp_off[q + 1] - grp_off[q];
            all_groups.push_back({q, tcount[q], nt, ns});
            if (ts_count[q] > 0) P->groups.push_back({q, tcount[q], ts_count[q], ns});
            n_pairs += nt * ns;
            sum_ns += (double)ns;
            ++n_busy;
        }
        P->list_hist = {n_busy ? sum_ns / n_busy : 0.0, n_busy ? (double)n_tgt / n_busy : 0.0};
        // conventional work: source slices per center, target chunks per center
        std::vector<ConvItem> conv_items;
        std::vector<ConvEvalItem> conv_eval;
        for (size_t i = 0; i < conv_centers.size(); ++i) {
            ConvCenter &cc = conv_centers[i];
            const int64_t ns = grp_off[cc.group + 1] - grp_off[cc.group];
            cc.part0 = (int32_t)conv_items.size();
            for (int64_t lo = 0; lo < ns || lo == 0; lo += kConvSlice) {
                conv_items.push_back(ConvItem{(int32_t)i, (int32_t)lo, (int32_t)std::min<int64_t>(ns, lo + kConvSlice),
                                              (int32_t)conv_items.size()});
                if (ns == 0) break;
            }
            cc.n_slices = (int32_t)conv_items.size() - cc.part0;
            for (int32_t j = 0; j < cc.n_tgt; j += 32)
                conv_eval.push_back(ConvEvalItem{(int32_t)i, cc.slot_begin + j, std::min<int32_t>(32, cc.n_tgt - j), 0});
        }

        // target slot records
        std::vector<double4_32a> slot_c(n_tgt), slot_e(n_tgt);
        std::vector<float4> slot_chi, slot_clo, slot_ef, slot_nf;
        std::vector<double4_32a> slot_n;
        if (mixed) { slot_chi.resize(n_tgt); slot_clo.resize(n_tgt); slot_ef.resize(n_tgt); }
        if (sp) { slot_n.resize(n_tgt); if (mixed) slot_nf.resize(n_tgt); }
        const int64_t nc = G->n_ctr;
        for (int64_t i = 0; i < n_tgt; ++i) {
            const int64_t t = slot_tgt[i];
            const int64_t c = G->tgt_center[t];
            double cc[3], e[3];
            for (int a = 0; a < 3; ++a) {
                cc[a] = G->ctr_xyz[a * nc + c];
                e[a] = G->tgt_xyz[a * n_tgt + t] - cc[a];
            }
            const double rho2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
            slot_c[i] = make_double4_32a(cc[0], cc[1], cc[2], 0.0);
            slot_e[i] = make_double4_32a(e[0], e[1], e[2], rho2);
            if (mixed) {
                float h[3], l[3];
                for (int a = 0; a < 3; ++a) split_ff(cc[a], h[a], l[a]);
                slot_chi[i] = make_float4(h[0], h[1], h[2], 0.f);
                slot_clo[i] = make_float4(l[0], l[1], l[2], 0.f);
                // -rho^2: the mixed kernels form -q2 directly (no sign operation per pair)
                slot_ef[i] = make_float4((float)e[0], (float)e[1], (float)e[2], (float)-rho2);
            }
            if (sp) {
                double nt[3];
                for (int a = 0; a < 3; ++a) nt[a] = G->tgt_normal[a * n_tgt + t];
                slot_n[i] = make_double4_32a(nt[0], nt[1], nt[2], 0.0);
                // the mixed S' kernels take -e.n_t, formed here in FP64
                if (mixed)
                    slot_nf[i] = make_float4((float)nt[0], (float)nt[1], (float)nt[2],
                                             (float)-(e[0] * nt[0] + e[1] * nt[1] + e[2] * nt[2]));
            }
        }
        // source records
        std::vector<double4_32a> src_pw(n_src), src_n;
        std::vector<float4> src_hi, src_lo, src_nf;
        if (dlp) src_n.resize(n_src);
        if (mixed) { src_hi.resize(n_src); src_lo.resize(n_src); if (dlp) src_nf.resize(n_src); }
        for (int64_t s = 0; s < n_src; ++s) {
            const double x = G->src_xyz[s], y = G->src_xyz[n_src + s], z = G->src_xyz[2 * n_src + s];
            src_pw[s] = make_double4_32a(x, y, z, G->src_weight[s]);
            if (dlp) {
                const double nx = G->src_normal[s], ny = G->src_normal[n_src + s],
                             nz = G->src_normal[2 * n_src + s];
                src_n[s] = make_double4_32a(nx, ny, nz, 0.0);
                // negated: the mixed double layer is formed from a' = -d.n_s, b' = -e.n_s
                if (mixed) src_nf[s] = make_float4((float)-nx, (float)-ny, (float)-nz, 0.f);
            }
            if (mixed) {
                float h[3], l[3];
                split_ff(x, h[0], l[0]); split_ff(y, h[1], l[1]); split_ff(z, h[2], l[2]);
                src_hi[s] = make_float4(h[0], h[1], h[2], 0.f);
                src_lo[s] = make_float4(l[0], l[1], l[2], 0.f);
            }
        }
        // upload geometry
        DevGeom &g = P->g;
        g.n_src = n_src;
        g.n_tgt = n_tgt;
        g.grp_off = P->upload(grp_off);
        g.grp_run = P->upload(grp_run);
        g.run_end = P->upload(run_end);
        g.run_src = P->upload(run_src);
        g.n_runs = (int32_t)run_end.size();
        g.src_pw = P->upload(src_pw);
        if (dlp) g.src_n = P->upload(src_n);
        if (mixed) {
            g.src_hi = P->upload(src_hi);
            g.src_lo = P->upload(src_lo);
            if (dlp) g.src_nf = P->upload(src_nf);
            g.slot_chi = P->upload(slot_chi);
            g.slot_clo = P->upload(slot_clo);
            g.slot_ef = P->upload(slot_ef);
            if (sp) g.slot_nf = P->upload(slot_nf);
        }
        if (sp) g.slot_n = P->upload(slot_n);
        g.slot_tgt = P->upload(slot_tgt);
        if (!conv_centers.empty()) {
            g.n_conv_centers = (int64_t)conv_centers.size();
            g.n_conv_items = (int64_t)conv_items.size();
            g.n_conv_eval = (int64_t)conv_eval.size();
            g.conv_centers = P->upload(conv_centers);
            g.conv_items = P->upload(conv_items);
            g.conv_eval = P->upload(conv_eval);
            P->conv_coef_doubles = (size_t)g.n_conv_items *
                                   (size_t)conv_coef_doubles(o->p, o->layers, o->kernel == TSQBX_HELMHOLTZ);
        }
        g.slot_c = P->upload(slot_c);
        g.slot_e = P->upload(slot_e);

        // evaluation slots (slot 0 serves tsqbx_eval / tsqbx_eval_async)
        const bool helm = o->kernel == TSQBX_HELMHOLTZ;
        P->density_bytes = (size_t)n_src * (helm ? 2 : 1) * sizeof(double);
        P->out_bytes = (size_t)n_tgt * (helm ? 2 : 1) * sizeof(double);
        P->wmu_bytes = (size_t)n_src * (helm ? sizeof(double2) : mixed ? sizeof(float) : sizeof(double));
        P->slots.resize(P->opt.n_slots + 1);
        const int prio = (o->flags & TSQBX_FLAG_SIZE_PRIORITY) ? size_priority(n_pairs, *o) : 0;
        for (auto &s : P->slots) {
            ck(cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio));
            ck(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
            // density, w mu, single- and double-layer buffers hold
            // rhs_capacity densities (tsqbx_submit_multi_layers), one after
            // another
            const size_t R = (size_t)rhs_capacity(*o);
            s.d_density = P->dalloc<char>(R * P->density_bytes);
            s.d_wmu = P->dalloc<char>(R * P->wmu_bytes);
            if (o->layers & TSQBX_SLP)
                s.d_out[0] = reinterpret_cast<double *>(P->dalloc<char>(R * P->out_bytes));
            if (o->layers & TSQBX_DLP)
                s.d_out[1] = reinterpret_cast<double *>(P->dalloc<char>(R * P->out_bytes));
            if (o->layers & TSQBX_SP) s.d_out[2] = reinterpret_cast<double *>(P->dalloc<char>(P->out_bytes));
            s.d_status = P->dalloc<int>(1);
            if (P->conv_coef_doubles) s.d_conv = P->dalloc<double>(P->conv_coef_doubles);
            s.h_density = P->halloc(R * P->density_bytes);
            s.h_out[0] = P->halloc(R * P->out_bytes);
            s.h_out[1] = P->halloc(R * P->out_bytes);
            if (o->layers & TSQBX_SP) s.h_out[2] = P->halloc(P->out_bytes);
            s.h_status = static_cast<int *>(P->halloc(sizeof(int)));
        }
        ck(cudaEventCreate(&P->k_begin));
        ck(cudaEventCreate(&P->k_end));

        // work schedule: options, else a cached tuning, else automatic
        int lanes = o->lanes_per_target;
        int64_t max_iters = o->max_item_iters;
        int tile = o->tile_depth ? o->tile_depth : kTile;
        int p_unroll = o->p_unroll, fp64_share = o->fp64_share;
        if ((o->flags & TSQBX_FLAG_USE_TUNED) && !lanes && !max_iters && !o->tile_depth && !o->p_unroll &&
            !o->fp64_share) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(tune_key(P));
            if (it != g_tune_cache.end()) {
                lanes = it->second.lanes_per_target;
                max_iters = it->second.max_item_iters;
                tile = it->second.tile_depth;
                p_unroll = it->second.p_unroll;
                fp64_share = it->second.fp64_share;
            }
        }
        P->g.tile = tile;
        P->g.p_unroll = p_unroll;
        P->g.fp64_share = fp64_share;
        Schedule sched;
        if ((rc = build_schedule(P->groups, lanes, max_iters, P->n_sm, sched, staging_weight(P))) != TSQBX_OK) {
            delete P;
            return rc;
        }
        apply_schedule(P, std::move(sched));

        // convergence check on the device, over every target (both paths)
        int64_t n_div = 0, n_zero = 0;
        if (!(o->flags & TSQBX_FLAG_SKIP_CHECK) && !all_groups.empty()) {
            Schedule chk;
            if ((rc = build_schedule(all_groups, 0, 0, P->n_sm, chk)) != TSQBX_OK) {
                delete P;
                return rc;
            }
            std::vector<Item> chk_items(chk.items.size());
            for (size_t i = 0; i < chk_items.size(); ++i) chk_items[i] = chk.items[i].it;
            DevGeom gc = g;
            gc.items = P->upload(chk_items);
            gc.n_items = (int64_t)chk_items.size();
            unsigned long long *cnt = P->dalloc<unsigned long long>(2);
            ck(cudaMemset(cnt, 0, 2 * sizeof(unsigned long long)));
            const int64_t blocks = (gc.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
            if (blocks > 0) check_pairs_kernel<<<(unsigned)blocks, kWarpsPerBlock * 32>>>(gc, cnt, cnt + 1);
            ck(cudaGetLastError());
            unsigned long long h[2] = {0, 0};
            ck(cudaMemcpy(h, cnt, sizeof(h), cudaMemcpyDeviceToHost));
            P->dfree(cnt);
            P->dfree(gc.items);
            n_div = (int64_t)h[0];
            n_zero = (int64_t)h[1];
            if (n_zero > 0 || (n_div > 0 && !(o->flags & TSQBX_FLAG_ALLOW_DIVERGENT))) {
                delete P;
                return TSQBX_E_DIVERGENT;
            }
        }

        tsqbx_plan_stats &st = P->stats;
        st.n_src = n_src;
        st.n_ctr = G->n_ctr;
        st.n_tgt = n_tgt;
        st.n_group = n_group;
        st.n_pairs = n_pairs;
        st.n_pair_terms = n_pairs * (int64_t)(o->p + 1);
        st.n_divergent = n_div;
        st.n_coincident = n_zero;
        st.list_entries = grp_off[n_group];
        st.n_conv_centers = g.n_conv_centers;
        st.n_conv_items = g.n_conv_items;
        for (const ConvCenter &cc : conv_centers) st.n_conv_targets += cc.n_tgt;
        fill_stats(P);
        *out = P;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        delete P;
        return status_of(f.err);
    } catch (const std::bad_alloc &) {
        delete P;
        return TSQBX_E_NOMEM;
    } catch (...) {
        delete P;
        return TSQBX_E_CUDA;
    }
}

void tsqbx_plan_destroy(tsqbx_plan P)
{
    if (!P) return;
    {
        std::lock_guard<std::mutex> lk(g_ticket_mu);
        for (auto it = g_tickets.begin(); it != g_tickets.end();)
            it = (it->second.first == P) ? g_tickets.erase(it) : std::next(it);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(P->opt.device);
    delete P;
    if (prev >= 0) cudaSetDevice(prev);
}

int tsqbx_plan_info(tsqbx_plan P, tsqbx_plan_stats *st)
{
    if (!P || !st) return TSQBX_E_INVAL;
    *st = P->stats;
    return TSQBX_OK;
}

int tsqbx_plan_kernel_ms(tsqbx_plan P, float *ms)
{
    if (!P || !ms || !P->k_timed) return TSQBX_E_INVAL;
    try {
        DeviceGuard dg(P->opt.device);
        cudaError_t e = cudaEventSynchronize(P->k_end);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, P->k_begin, P->k_end);
        if (e != cudaSuccess) { cudaGetLastError(); return status_of(e); }
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    }
}

int tsqbx_plan_footprint(tsqbx_plan P, size_t *bytes)
{
    if (!P || !bytes) return TSQBX_E_INVAL;
    *bytes = P->device_bytes;
    return TSQBX_OK;
}

int tsqbx_plan_get_tuning(tsqbx_plan P, tsqbx_tuning *t)
{
    if (!P || !t) return TSQBX_E_INVAL;
    t->lanes_per_target = P->sched.lanes_policy;
    t->max_item_iters = (int)P->sched.max_iters;
    t->kernel_ms = 0.f;
    t->tile_depth = P->g.tile;
    t->p_unroll = P->g.p_unroll;
    t->fp64_share = P->g.fp64_share;
    return TSQBX_OK;
}

int tsqbx_plan_set_tuning(tsqbx_plan P, const tsqbx_tuning *t)
{
    if (!P || !t || t->lanes_per_target < 0 || t->lanes_per_target > 32 || t->max_item_iters < 0 ||
        (t->tile_depth != 0 && !tile_depth_ok(t->tile_depth)) || !p_unroll_ok(t->p_unroll) ||
        t->fp64_share < 0 || t->fp64_share > 20)
        return TSQBX_E_INVAL;
    if (t->p_unroll != 0 && !has_runtime_order(P->opt.kernel, P->opt.precision)) return TSQBX_E_UNSUPPORTED;
    if (t->fp64_share != 0 && !has_both_pipes(P->opt.kernel, P->opt.precision)) return TSQBX_E_UNSUPPORTED;
    try {
        DeviceGuard dg(P->opt.device);
        std::lock_guard<std::mutex> lk(P->mu);
        for (Slot &s : P->slots) ck(cudaStreamSynchronize(s.stream));
        Schedule sched;
        int rc = build_schedule(P->groups, t->lanes_per_target, t->max_item_iters, P->n_sm, sched,
                                staging_weight(P));
        if (rc) return rc;
        apply_schedule(P, std::move(sched));
        P->g.tile = t->tile_depth ? t->tile_depth : kTile;
        P->g.p_unroll = t->p_unroll;
        P->g.fp64_share = t->fp64_share;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    } catch (const std::bad_alloc &) {
        return TSQBX_E_NOMEM;
    }
}

int tsqbx_plan_autotune(tsqbx_plan P, const void *d_density, int repeats, tsqbx_tuning *chosen)
{
    if (!P || (P->g.n_src && !d_density) || repeats < 1) return TSQBX_E_INVAL;
    try {
        DeviceGuard dg(P->opt.device);
        std::lock_guard<std::mutex> lk(P->mu);
        Slot &slot = P->slots[0];
        for (Slot &s : P->slots) ck(cudaStreamSynchronize(s.stream));
        auto time_current = [&](float &median_ms) -> int {
            float acc[64];
            const int reps = std::min(repeats, 64);
            for (int r = -1; r < reps; ++r) {
                int rc = enqueue(P, slot, d_density, slot.d_out[0], slot.d_out[1], slot.d_out[2], slot.stream, true,
                                 P->opt.p, P->opt.k);
                if (rc) return rc;
                ck(cudaEventSynchronize(P->k_end));
                float ms = 0.f;
                ck(cudaEventElapsedTime(&ms, P->k_begin, P->k_end));
                if (r >= 0) acc[r] = ms;
            }
            std::sort(acc, acc + reps);
            median_ms = acc[reps / 2];
            return TSQBX_OK;
        };
        struct Cand { int lanes; int64_t iters; int tile; int unroll; int share; float ms; };
        Cand best{P->sched.lanes_policy, P->sched.max_iters, P->g.tile, P->g.p_unroll, P->g.fp64_share, 0.f};
        int rc = time_current(best.ms);
        if (rc) return rc;
        auto trial = [&](int lanes, int64_t iters, int tile, int unroll, int share) -> int {
            Schedule sched;
            int r = build_schedule(P->groups, lanes, iters, P->n_sm, sched, staging_weight(P));
            if (r) return r;
            apply_schedule(P, std::move(sched));
            P->g.tile = tile;
            P->g.p_unroll = unroll;
            P->g.fp64_share = share;
            float ms = 0.f;
            if ((r = time_current(ms)) != TSQBX_OK) return r;
            if (ms < best.ms) best = {lanes, P->sched.max_iters, tile, unroll, share, ms};
            return TSQBX_OK;
        };
        // stage 1: slice caps with the current lane policy, depth and order
        // form; stage 2: lane policies at the best cap; stage 3: tile depths at
        // both; stage 4 (Laplace FP64 and mixed): the order-loop forms
        for (int64_t iters : {64, 128, 256, 512, 1024, 2048})
            if ((rc = trial(best.lanes, iters, best.tile, best.unroll, best.share)) != TSQBX_OK) return rc;
        const int64_t cap = best.iters;
        for (int lanes : {0, 1, 2, 4, 8, 16})
            if ((rc = trial(lanes, cap, best.tile, best.unroll, best.share)) != TSQBX_OK) return rc;
        const int lanes_best = best.lanes;
        for (int tile : {kTileMin, kTile, kTileMax})
            if ((rc = trial(lanes_best, cap, tile, best.unroll, best.share)) != TSQBX_OK) return rc;
        const int tile_best = best.tile;
        if (has_runtime_order(P->opt.kernel, P->opt.precision))
            for (int unroll : {0, 1, 2, 4})
                if ((rc = trial(lanes_best, cap, tile_best, unroll, best.share)) != TSQBX_OK) return rc;
        if (has_both_pipes(P->opt.kernel, P->opt.precision))
            for (int share : {0, 1, 2, 3})
                if ((rc = trial(lanes_best, cap, tile_best, best.unroll, share)) != TSQBX_OK) return rc;
        Schedule sched;
        if ((rc = build_schedule(P->groups, best.lanes, best.iters, P->n_sm, sched, staging_weight(P))) !=
            TSQBX_OK)
            return rc;
        apply_schedule(P, std::move(sched));
        P->g.tile = best.tile;
        P->g.p_unroll = best.unroll;
        P->g.fp64_share = best.share;
        tsqbx_tuning t{best.lanes, (int)best.iters, best.ms, best.tile, best.unroll, best.share};
        {
            std::lock_guard<std::mutex> tl(g_tune_mu);
            g_tune_cache[tune_key(P)] = t;
        }
        if (chosen) *chosen = t;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    } catch (const std::bad_alloc &) {
        return TSQBX_E_NOMEM;
    }
}

}  // extern "C"

namespace {

bool pk_ok(tsqbx_plan P, int p, double k)
{
    if (p < 0 || p > TSQBX_P_MAX) return false;
    return P->opt.kernel != TSQBX_HELMHOLTZ || (k > 0.0 && std::isfinite(k));
}

bool layer_args_ok(tsqbx_plan P, const void *out_slp, const void *out_dlp)
{
    if ((P->opt.layers & TSQBX_SLP) && !out_slp && P->g.n_tgt) return false;
    if ((P->opt.layers & TSQBX_DLP) && !out_dlp && P->g.n_tgt) return false;
    return true;
}

// Stage inputs, enqueue, and (for host outputs) copy back into pinned
// staging; records slot.done.  Host outputs are delivered by finish().
int start(tsqbx_plan P, Slot &slot, const void *density, void *out_slp, void *out_dlp, void *out_sp,
          bool timed, int p, double k)
{
    const void *d_density = density;
    if (P->g.n_src && !is_device_ptr(density)) {
        std::memcpy(slot.h_density, density, P->density_bytes);
        ck(cudaMemcpyAsync(slot.d_density, slot.h_density, P->density_bytes, cudaMemcpyHostToDevice,
                           slot.stream));
        d_density = slot.d_density;
    }
    void *outs[3] = {out_slp, out_dlp, out_sp};
    double *d_outs[3] = {nullptr, nullptr, nullptr};
    reset_multi(slot);
    for (int l = 0; l < 3; ++l) {
        slot.user_out[l] = outs[l];
        slot.copy_out[l] = false;
        if (!outs[l] || !slot.d_out[l]) continue;
        if (is_device_ptr(outs[l])) d_outs[l] = static_cast<double *>(outs[l]);
        else { d_outs[l] = slot.d_out[l]; slot.copy_out[l] = true; }
    }
    ck(cudaMemsetAsync(slot.d_status, 0, sizeof(int), slot.stream));
    int rc = enqueue(P, slot, d_density, d_outs[0], d_outs[1], d_outs[2], slot.stream, timed, p, k);
    if (rc) return rc;
    for (int l = 0; l < 3; ++l)
        if (slot.copy_out[l] && P->out_bytes)
            ck(cudaMemcpyAsync(slot.h_out[l], slot.d_out[l], P->out_bytes, cudaMemcpyDeviceToHost,
                               slot.stream));
    ck(cudaMemcpyAsync(slot.h_status, slot.d_status, sizeof(int), cudaMemcpyDeviceToHost, slot.stream));
    ck(cudaEventRecord(slot.done, slot.stream));
    return TSQBX_OK;
}

// The same for n densities of a multi-density plan (tsqbx_submit_multi_layers):
// host densities are staged one after another in the slot's buffers, host
// outputs come back through the slot's single- and double-layer staging.
// outs[0] / outs[1]: the single- / double-layer outputs (arrays of n
// pointers; read only for the layers of the plan's mask).
int start_multi(tsqbx_plan P, Slot &slot, int n, const void *const *density, void *const *const (&outs)[2], int p,
                double k)
{
    const void *dens[kMaxRhs];
    for (int r = 0; r < n; ++r) {
        dens[r] = density[r];
        if (P->g.n_src && !is_device_ptr(density[r])) {
            char *h = static_cast<char *>(slot.h_density) + (size_t)r * P->density_bytes;
            char *d = static_cast<char *>(slot.d_density) + (size_t)r * P->density_bytes;
            std::memcpy(h, density[r], P->density_bytes);
            ck(cudaMemcpyAsync(d, h, P->density_bytes, cudaMemcpyHostToDevice, slot.stream));
            dens[r] = d;
        }
    }
    double *d_outs[2][kMaxRhs] = {};
    const uint32_t mask[2] = {TSQBX_SLP, TSQBX_DLP};
    slot.n_rhs = n;
    for (int l = 0; l < 3; ++l) {
        slot.user_out[l] = nullptr;
        slot.copy_out[l] = false;
    }
    for (int l = 0; l < 2; ++l) {
        if (!(P->opt.layers & mask[l])) continue;
        for (int r = 0; r < n; ++r) {
            slot.user_out_rhs[l][r] = outs[l][r];
            slot.copy_out_rhs[l][r] = !is_device_ptr(outs[l][r]);
            d_outs[l][r] = slot.copy_out_rhs[l][r] ? slot.d_out[l] + (size_t)r * (P->out_bytes / sizeof(double))
                                                   : static_cast<double *>(outs[l][r]);
        }
    }
    ck(cudaMemsetAsync(slot.d_status, 0, sizeof(int), slot.stream));
    int rc = enqueue_multi(P, slot, n, nullptr, dens, d_outs, slot.stream, p, k);
    if (rc) return rc;
    for (int l = 0; l < 2; ++l)
        for (int r = 0; r < n; ++r)
            if (slot.copy_out_rhs[l][r] && P->out_bytes)
                ck(cudaMemcpyAsync(static_cast<char *>(slot.h_out[l]) + (size_t)r * P->out_bytes, d_outs[l][r],
                                   P->out_bytes, cudaMemcpyDeviceToHost, slot.stream));
    ck(cudaMemcpyAsync(slot.h_status, slot.d_status, sizeof(int), cudaMemcpyDeviceToHost, slot.stream));
    ck(cudaEventRecord(slot.done, slot.stream));
    return TSQBX_OK;
}

int finish(tsqbx_plan P, Slot &slot)
{
    for (int l = 0; l < 3; ++l)
        if (slot.copy_out[l]) std::memcpy(slot.user_out[l], slot.h_out[l], P->out_bytes);
    for (int l = 0; l < 2; ++l)                   // outputs of a multi-density call
        for (int r = 0; r < slot.n_rhs; ++r)
            if (slot.copy_out_rhs[l][r])
                std::memcpy(slot.user_out_rhs[l][r],
                            static_cast<char *>(slot.h_out[l]) + (size_t)r * P->out_bytes, P->out_bytes);
    reset_multi(slot);
    return *slot.h_status ? TSQBX_E_KERNEL : TSQBX_OK;
}

}  // namespace

extern "C" {

int tsqbx_eval_pk(tsqbx_plan P, int p, double k, const void *density, void *out_slp, void *out_dlp,
                  void *out_sp)
{
    if (!P || (P->g.n_src && !density) || !layer_args_ok(P, out_slp, out_dlp) || !pk_ok(P, p, k))
        return TSQBX_E_INVAL;
    try {
        DeviceGuard dg(P->opt.device);
        std::lock_guard<std::mutex> lk(P->mu);
        Slot &slot = P->slots[0];
        int rc = start(P, slot, density, out_slp, out_dlp, out_sp, true, p, k);
        if (rc) return rc;
        ck(cudaEventSynchronize(slot.done));
        return finish(P, slot);
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    } catch (...) {
        return TSQBX_E_CUDA;
    }
}

int tsqbx_eval(tsqbx_plan P, const void *density, void *out_slp, void *out_dlp)
{
    if (!P) return TSQBX_E_INVAL;
    return tsqbx_eval_pk(P, P->opt.p, P->opt.k, density, out_slp, out_dlp, nullptr);
}

int tsqbx_eval_async_pk(tsqbx_plan P, int p, double k, const void *d_density, void *d_out_slp, void *d_out_dlp,
                        void *d_out_sp, void *stream)
{
    if (!P || (P->g.n_src && !d_density) || !layer_args_ok(P, d_out_slp, d_out_dlp) || !pk_ok(P, p, k))
        return TSQBX_E_INVAL;
    try {
        DeviceGuard dg(P->opt.device);
        Slot &slot = P->slots[0];
        cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : slot.stream;
        return enqueue(P, slot, d_density, static_cast<double *>(d_out_slp), static_cast<double *>(d_out_dlp),
                       static_cast<double *>(d_out_sp), s, true, p, k);
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    } catch (...) {
        return TSQBX_E_CUDA;
    }
}

int tsqbx_eval_async(tsqbx_plan P, const void *d_density, void *d_out_slp, void *d_out_dlp, void *stream)
{
    if (!P) return TSQBX_E_INVAL;
    return tsqbx_eval_async_pk(P, P->opt.p, P->opt.k, d_density, d_out_slp, d_out_dlp, nullptr, stream);
}

int tsqbx_submit_pk(tsqbx_plan P, int p, double k, const void *density, void *out_slp, void *out_dlp,
                    void *out_sp, uint64_t *ticket)
{
    if (!P || !ticket || (P->g.n_src && !density) || !layer_args_ok(P, out_slp, out_dlp) || !pk_ok(P, p, k))
        return TSQBX_E_INVAL;
    try {
        DeviceGuard dg(P->opt.device);
        std::lock_guard<std::mutex> lk(P->mu);
        int idx = -1;
        for (size_t i = 1; i < P->slots.size(); ++i)
            if (!P->slots[i].busy) { idx = (int)i; break; }
        if (idx < 0) return TSQBX_E_BUSY;
        Slot &slot = P->slots[idx];
        int rc = start(P, slot, density, out_slp, out_dlp, out_sp, false, p, k);
        if (rc) return rc;
        slot.busy = true;
        slot.ticket = g_next_ticket.fetch_add(1);
        {
            std::lock_guard<std::mutex> tl(g_ticket_mu);
            g_tickets[slot.ticket] = {P, idx};
        }
        *ticket = slot.ticket;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    } catch (...) {
        return TSQBX_E_CUDA;
    }
}

int tsqbx_submit_multi_layers(tsqbx_plan P, int p, double k, int n, const void *const *density,
                              void *const *out_slp, void *const *out_dlp, uint64_t *ticket)
{
    if (!P || !ticket || !density || n < 1 || n > rhs_capacity(P->opt) || !pk_ok(P, p, k)) return TSQBX_E_INVAL;
    if (!multi_ok(P->opt) || P->g.n_conv_centers > 0) return TSQBX_E_UNSUPPORTED;
    const bool slp = (P->opt.layers & TSQBX_SLP) != 0, dlp = (P->opt.layers & TSQBX_DLP) != 0;
    if ((slp && !out_slp) || (dlp && !out_dlp)) return TSQBX_E_INVAL;
    for (int r = 0; r < n; ++r)
        if ((P->g.n_src && !density[r]) || (P->g.n_tgt && ((slp && !out_slp[r]) || (dlp && !out_dlp[r]))))
            return TSQBX_E_INVAL;
    try {
        DeviceGuard dg(P->opt.device);
        std::lock_guard<std::mutex> lk(P->mu);
        int idx = -1;
        for (size_t i = 1; i < P->slots.size(); ++i)
            if (!P->slots[i].busy) { idx = (int)i; break; }
        if (idx < 0) return TSQBX_E_BUSY;
        Slot &slot = P->slots[idx];
        void *const *const outs[2] = {out_slp, out_dlp};
        int rc = start_multi(P, slot, n, density, outs, p, k);
        if (rc) {
            reset_multi(slot);
            return rc;
        }
        slot.busy = true;
        slot.ticket = g_next_ticket.fetch_add(1);
        {
            std::lock_guard<std::mutex> tl(g_ticket_mu);
            g_tickets[slot.ticket] = {P, idx};
        }
        *ticket = slot.ticket;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    } catch (...) {
        return TSQBX_E_CUDA;
    }
}

int tsqbx_submit_multi(tsqbx_plan P, int p, double k, int n, const void *const *density, void *const *out_slp,
                       uint64_t *ticket)
{
    return tsqbx_submit_multi_layers(P, p, k, n, density, out_slp, nullptr, ticket);
}

int tsqbx_submit(tsqbx_plan P, const void *density, void *out_slp, void *out_dlp, uint64_t *ticket)
{
    if (!P) return TSQBX_E_INVAL;
    return tsqbx_submit_pk(P, P->opt.p, P->opt.k, density, out_slp, out_dlp, nullptr, ticket);
}

int tsqbx_poll(uint64_t ticket, int timeout_us)
{
    tsqbx_plan P = nullptr;
    int idx = -1;
    {
        std::lock_guard<std::mutex> tl(g_ticket_mu);
        auto it = g_tickets.find(ticket);
        if (it == g_tickets.end()) return TSQBX_E_NOTFOUND;
        P = it->second.first;
        idx = it->second.second;
    }
    try {
        DeviceGuard dg(P->opt.device);
        Slot &slot = P->slots[idx];
        cudaError_t q = cudaEventQuery(slot.done);
        if (q == cudaErrorNotReady) {
            if (timeout_us == 0) return TSQBX_PENDING;
            if (timeout_us < 0) {
                q = cudaEventSynchronize(slot.done);
            } else {
                const auto t_end = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
                while ((q = cudaEventQuery(slot.done)) == cudaErrorNotReady) {
                    if (std::chrono::steady_clock::now() >= t_end) return TSQBX_E_TIMEOUT;
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                }
            }
        }
        std::lock_guard<std::mutex> lk(P->mu);
        {
            std::lock_guard<std::mutex> tl(g_ticket_mu);
            if (!g_tickets.erase(ticket)) return TSQBX_E_NOTFOUND;
        }
        int rc;
        if (q != cudaSuccess) {
            cudaGetLastError();
            rc = status_of(q);
        } else {
            rc = finish(P, slot);
        }
        slot.busy = false;
        return rc;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        return status_of(f.err);
    } catch (...) {
        return TSQBX_E_CUDA;
    }
}

}  // extern "C"
