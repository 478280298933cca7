// server.cu -- a request-serving runtime over libtsqbx plans.
//
// Requests (an evaluation of one registered geometry with a kernel variant
// and a density) arrive at any time.  A worker thread keeps them moving:
//  * admission: a queued request is started as soon as its plan (geometry,
//    kernel, layers, p, k, precision) is resident with a free slot and the
//    resident plans fit the HBM budget -- plans are created on first use, and
//    idle plans are evicted least-recently-used when the budget would be
//    exceeded;
//  * continuous batching: every started request runs on its own plan slot
//    (own stream), so requests that arrive while others are on the GPU overlap
//    with them; completions free slots for the next queued requests.  Queued
//    requests (Helmholtz single layer; Laplace single and/or double layer in
//    FP64 or double-float) that share a plan, an order and (Helmholtz) a
//    wavenumber start together as one multi-density evaluation
//    (tsqbx_submit_multi_layers), which costs little more than one of them;
//  * accounting: latency (arrival to completion) per request, p50/p99,
//    pair-terms completed, plans created/evicted, resident bytes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "plan_internal.h"

using namespace tsqbx;

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) { return std::chrono::duration<double>(Clock::now() - t0).count(); }

// Host copy of a registered geometry.
struct GeomCopy {
    std::vector<double> src_xyz, src_weight, src_normal, ctr_xyz, ctr_radius, tgt_xyz, tgt_normal;
    std::vector<int32_t> tgt_center, ctr_group, range_begin, range_end;
    std::vector<int64_t> group_range_start;
    tsqbx_geometry view{};
};

using PlanKey = std::tuple<int, int, unsigned, int>;   // geom, kernel, layers, precision

struct PlanEntry {
    tsqbx_plan plan = nullptr;
    size_t bytes = 0;
    int inflight = 0;
    uint64_t last_use = 0;
};

enum class RState { Queued, Running, Done };

struct Request {
    uint64_t id = 0;
    int geom = 0;
    tsqbx_options opt{};
    PlanKey key;
    std::vector<double> density;
    void *out_slp = nullptr, *out_dlp = nullptr, *out_sp = nullptr;
    Clock::time_point arrive;
    double latency_s = 0;
    RState state = RState::Queued;
    int status = TSQBX_OK;
    uint64_t ticket = 0;
    int64_t pair_terms = 0;
    std::vector<Request *> merged;   // queued requests that ride in this one's evaluation
};

// Densities one evaluation of the server may carry: queued requests with the
// same plan, order and (Helmholtz) wavenumber are started together
// (tsqbx_submit_multi_layers) when a slot frees up.
constexpr int kServerMaxRhs = 4;

// The plans tsqbx_submit_multi_layers takes -- Helmholtz single layer;
// Laplace single and/or double layer in FP64 or double-float -- without
// conventional centers.
bool mergeable(const tsqbx_options &o)
{
    const bool laplace_ok = o.kernel == TSQBX_LAPLACE && o.precision != TSQBX_MIXED && o.layers != 0 &&
                            !(o.layers & ~(uint32_t)(TSQBX_SLP | TSQBX_DLP));
    return (laplace_ok || (o.kernel == TSQBX_HELMHOLTZ && o.layers == TSQBX_SLP)) &&
           !(o.flags & (TSQBX_FLAG_CONVENTIONAL_AUTO | TSQBX_FLAG_CONVENTIONAL_ALL));
}

size_t estimate_bytes(const GeomCopy &g, const tsqbx_options &o)
{
    // the larger device arrays of a plan (sources, list runs, target slots,
    // slot buffers); the ranges bound the merged runs (8 bytes each)
    const size_t ns = (size_t)g.view.n_src, nt = (size_t)g.view.n_tgt;
    const bool helm = o.kernel == TSQBX_HELMHOLTZ, mixed = o.precision == TSQBX_MIXED;
    size_t b = ns * 32 + g.range_begin.size() * 8 + nt * (4 + 64) + (size_t)g.view.n_group * 12;
    if (o.layers & TSQBX_DLP) b += ns * 32;
    if (o.layers & TSQBX_SP) b += nt * 32;
    if (mixed) b += ns * 48 + nt * 48;
    const int slots = (o.n_slots ? o.n_slots : 2) + 1;
    const size_t rhs = o.max_rhs > 1 ? (size_t)o.max_rhs : 1;
    b += (size_t)slots * rhs *
         (ns * (helm ? 32 : 16) + nt * 16 * (helm ? 2 : 1) + ((o.layers & TSQBX_DLP) ? nt * 16 : 0));
    return b;
}

}  // namespace

struct tsqbx_server_s {
    int device = 0;
    size_t budget = 0;
    bool size_priority = false;              // plans built with TSQBX_FLAG_SIZE_PRIORITY
    bool laplace_fp64_as_df64 = false;       // Laplace FP64 requests served by DF64 plans
    int max_inflight = 64;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    std::vector<std::unique_ptr<GeomCopy>> geoms;
    std::map<PlanKey, PlanEntry> plans;
    std::map<PlanKey, size_t> known_bytes;   // exact footprints of plans built before
    std::list<Request *> queue;
    std::vector<Request *> running;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
    uint64_t next_id = 1, use_clock = 0;
    size_t resident = 0;
    std::vector<double> lat;                 // seconds, completed requests
    int64_t completed = 0, failed = 0, rejected = 0, created = 0, evicted = 0, pair_terms = 0, merged = 0;
    Clock::time_point t_first{}, t_last{};
    bool any_done = false, span_started = false;

    void run();
    bool admit(Request *r);
    void evict_for(size_t need, const PlanKey *keep = nullptr);
};

// Evict idle plans, least recently used first, until `need` more bytes fit
// (never the plan `keep`, e.g. the one being admitted).
void tsqbx_server_s::evict_for(size_t need, const PlanKey *keep)
{
    while (resident + need > budget) {
        auto victim = plans.end();
        for (auto it = plans.begin(); it != plans.end(); ++it)
            if (it->second.inflight == 0 && !(keep && it->first == *keep) &&
                (victim == plans.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == plans.end()) return;
        resident -= victim->second.bytes;
        tsqbx_plan_destroy(victim->second.plan);
        plans.erase(victim);
        ++evicted;
    }
}

// Try to start one queued request; false if it has to wait (memory or slots).
bool tsqbx_server_s::admit(Request *r)
{
    auto it = plans.find(r->key);
    if (it == plans.end()) {
        const GeomCopy &g = *geoms[r->geom];
        auto kb = known_bytes.find(r->key);
        const size_t need = kb != known_bytes.end() ? kb->second : estimate_bytes(g, r->opt);
        if (need > budget) {                                   // can never fit
            r->status = TSQBX_E_NOMEM;
            return true;
        }
        if (resident + need > budget) evict_for(need);
        if (resident + need > budget) return false;            // wait for running work
        tsqbx_plan P = nullptr;
        int rc = tsqbx_plan_create(&g.view, &r->opt, &P);
        if (rc != TSQBX_OK) {
            r->status = rc;
            return true;
        }
        size_t bytes = 0;
        tsqbx_plan_footprint(P, &bytes);
        known_bytes[r->key] = bytes;
        if (resident + bytes > budget) evict_for(bytes);       // the estimate was low
        if (resident + bytes > budget) {                       // still no room: retry later
            tsqbx_plan_destroy(P);
            if (bytes > budget) r->status = TSQBX_E_NOMEM;
            return bytes > budget;
        }
        it = plans.emplace(r->key, PlanEntry{P, bytes, 0, ++use_clock}).first;
        resident += bytes;
        ++created;
    }
    PlanEntry &pe = it->second;
    // queued requests for the same plan, order and wavenumber ride along
    std::vector<Request *> group{r};
    if (r->opt.max_rhs > 1)
        for (Request *q : queue) {
            if ((int)group.size() >= r->opt.max_rhs) break;
            if (q != r && q->state == RState::Queued && q->key == r->key && q->opt.p == r->opt.p &&
                (r->opt.kernel == TSQBX_LAPLACE || q->opt.k == r->opt.k))
                group.push_back(q);
        }
    int rc;
    if (group.size() > 1) {
        const void *dens[kServerMaxRhs];
        void *outs[kServerMaxRhs], *outs_dlp[kServerMaxRhs];
        for (size_t i = 0; i < group.size(); ++i) {
            dens[i] = group[i]->density.data();
            outs[i] = group[i]->out_slp;
            outs_dlp[i] = group[i]->out_dlp;
        }
        rc = tsqbx_submit_multi_layers(pe.plan, r->opt.p, r->opt.k, (int)group.size(), dens, outs, outs_dlp,
                                       &r->ticket);
    } else {
        rc = tsqbx_submit_pk(pe.plan, r->opt.p, r->opt.k, r->density.data(), r->out_slp, r->out_dlp, r->out_sp,
                             &r->ticket);
    }
    if (rc == TSQBX_E_BUSY) return false;                      // every slot of the plan busy
    if (rc != TSQBX_OK) {
        r->status = rc;
        return true;
    }
    tsqbx_plan_stats st{};
    tsqbx_plan_info(pe.plan, &st);
    r->pair_terms = st.n_pairs * (int64_t)(r->opt.p + 1);
    for (size_t i = 1; i < group.size(); ++i) {
        Request *q = group[i];
        q->state = RState::Running;
        q->pair_terms = r->pair_terms;
        r->merged.push_back(q);
        queue.remove(q);
    }
    ++pe.inflight;
    pe.last_use = ++use_clock;
    r->state = RState::Running;
    running.push_back(r);
    return true;
}

void tsqbx_server_s::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        bool progressed = false;
        // completions
        for (size_t i = 0; i < running.size();) {
            Request *r = running[i];
            const int rc = tsqbx_poll(r->ticket, 0);
            if (rc == TSQBX_PENDING) { ++i; continue; }
            auto pit = plans.find(r->key);
            if (pit != plans.end()) --pit->second.inflight;
            merged += (int64_t)r->merged.size();
            std::vector<Request *> done{r};
            done.insert(done.end(), r->merged.begin(), r->merged.end());
            for (Request *d : done) {
                d->latency_s = seconds_since(d->arrive);
                d->status = rc;
                d->state = RState::Done;
                if (rc == TSQBX_OK) {
                    ++completed;
                    pair_terms += d->pair_terms;
                    lat.push_back(d->latency_s);
                } else {
                    ++failed;
                }
            }
            t_last = Clock::now();
            any_done = true;
            running[i] = running.back();
            running.pop_back();
            progressed = true;
        }
        // admissions, in arrival order; a waiting request does not block
        // later requests whose plans are free
        for (auto qit = queue.begin(); qit != queue.end() && (int)running.size() < max_inflight;) {
            Request *r = *qit;
            if (!admit(r)) { ++qit; continue; }
            if (r->state != RState::Running) {                 // admission failed for good
                r->state = RState::Done;
                r->latency_s = seconds_since(r->arrive);
                ++rejected;
            }
            qit = queue.erase(qit);
            progressed = true;
        }
        if (progressed) cv.notify_all();
        if (running.empty() && queue.empty()) cv.wait(lk, [&] { return stop || !queue.empty(); });
        else if (!progressed) cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

extern "C" {

int tsqbx_server_create(int device, size_t hbm_budget_bytes, int max_inflight, tsqbx_server *out)
{
    if (!out || device < 0 || max_inflight < 1 || hbm_budget_bytes == 0) return TSQBX_E_INVAL;
    *out = nullptr;
    tsqbx_server S = new (std::nothrow) tsqbx_server_s;
    if (!S) return TSQBX_E_NOMEM;
    S->device = device;
    S->budget = hbm_budget_bytes;
    S->max_inflight = max_inflight;
    try {
        S->worker = std::thread([S] { S->run(); });
    } catch (...) {
        delete S;
        return TSQBX_E_NOMEM;
    }
    *out = S;
    return TSQBX_OK;
}

void tsqbx_server_destroy(tsqbx_server S)
{
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // let running work finish so no kernel writes into freed buffers
        S->cv.wait(lk, [&] { return S->running.empty(); });
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->plans) tsqbx_plan_destroy(kv.second.plan);
    delete S;
}

int tsqbx_server_add_geometry(tsqbx_server S, const tsqbx_geometry *G, int *geom_id)
{
    if (!S || !G || !geom_id || G->n_src < 0 || G->n_ctr < 0 || G->n_tgt < 0 || G->n_group < 0 ||
        !G->group_range_start)
        return TSQBX_E_INVAL;
    try {
        auto g = std::make_unique<GeomCopy>();
        auto cp = [](auto *src, int64_t n, auto &dst) {
            if (src && n > 0) dst.assign(src, src + n);
        };
        const int64_t nnz = G->group_range_start[G->n_group];
        cp(G->src_xyz, 3 * G->n_src, g->src_xyz);
        cp(G->src_weight, G->n_src, g->src_weight);
        cp(G->src_normal, 3 * G->n_src, g->src_normal);
        cp(G->ctr_xyz, 3 * G->n_ctr, g->ctr_xyz);
        cp(G->ctr_radius, G->n_ctr, g->ctr_radius);
        cp(G->tgt_xyz, 3 * G->n_tgt, g->tgt_xyz);
        cp(G->tgt_normal, 3 * G->n_tgt, g->tgt_normal);
        cp(G->tgt_center, G->n_tgt, g->tgt_center);
        cp(G->ctr_group, G->n_ctr, g->ctr_group);
        cp(G->group_range_start, G->n_group + 1, g->group_range_start);
        cp(G->range_begin, nnz, g->range_begin);
        cp(G->range_end, nnz, g->range_end);
        auto ptr = [](auto &v) { return v.empty() ? nullptr : v.data(); };
        g->view = tsqbx_geometry{G->n_src, ptr(g->src_xyz), ptr(g->src_weight), ptr(g->src_normal),
                                 G->n_ctr, ptr(g->ctr_xyz), ptr(g->ctr_radius), G->n_tgt, ptr(g->tgt_xyz),
                                 ptr(g->tgt_center), G->n_group, ptr(g->ctr_group),
                                 g->group_range_start.data(), ptr(g->range_begin), ptr(g->range_end),
                                 ptr(g->tgt_normal)};
        std::lock_guard<std::mutex> lk(S->mu);
        S->geoms.push_back(std::move(g));
        *geom_id = (int)S->geoms.size() - 1;
        return TSQBX_OK;
    } catch (const std::bad_alloc &) {
        return TSQBX_E_NOMEM;
    }
}

int tsqbx_server_submit(tsqbx_server S, int geom_id, const tsqbx_options *opt, const void *density,
                        void *out_slp, void *out_dlp, void *out_sp, uint64_t *request)
{
    if (!S || !opt || !request) return TSQBX_E_INVAL;
    try {
        auto r = std::make_unique<Request>();
        r->arrive = Clock::now();
        std::unique_lock<std::mutex> lk(S->mu);
        if (geom_id < 0 || geom_id >= (int)S->geoms.size()) return TSQBX_E_INVAL;
        const GeomCopy &g = *S->geoms[geom_id];
        const int64_t width = opt->kernel == TSQBX_HELMHOLTZ ? 2 : 1;
        if (g.view.n_src && !density) return TSQBX_E_INVAL;
        if (((opt->layers & TSQBX_SLP) && g.view.n_tgt && !out_slp) ||
            ((opt->layers & TSQBX_DLP) && g.view.n_tgt && !out_dlp) ||
            ((opt->layers & TSQBX_SP) && g.view.n_tgt && !out_sp))
            return TSQBX_E_INVAL;
        r->id = S->next_id++;
        r->geom = geom_id;
        r->opt = *opt;
        if (S->size_priority) r->opt.flags |= TSQBX_FLAG_SIZE_PRIORITY;
        if (S->laplace_fp64_as_df64 && r->opt.kernel == TSQBX_LAPLACE && r->opt.precision == TSQBX_FP64)
            r->opt.precision = TSQBX_DF64;
        if (mergeable(r->opt)) r->opt.max_rhs = kServerMaxRhs;
        r->opt.device = S->device;
        r->key = PlanKey{geom_id, (int)r->opt.kernel, r->opt.layers, (int)r->opt.precision};
        const double *d = static_cast<const double *>(density);
        if (d) r->density.assign(d, d + g.view.n_src * width);
        r->out_slp = out_slp;
        r->out_dlp = out_dlp;
        r->out_sp = out_sp;
        if (!S->span_started) {
            S->t_first = r->arrive;
            S->span_started = true;
        }
        *request = r->id;
        S->queue.push_back(r.get());
        S->requests.emplace(r->id, std::move(r));
        lk.unlock();
        S->cv.notify_all();
        return TSQBX_OK;
    } catch (const std::bad_alloc &) {
        return TSQBX_E_NOMEM;
    }
}

int tsqbx_server_poll(tsqbx_server S, uint64_t request, int timeout_us)
{
    if (!S) return TSQBX_E_INVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(request);
    if (it == S->requests.end()) return TSQBX_E_NOTFOUND;
    Request *r = it->second.get();
    auto done = [&] { return r->state == RState::Done; };
    if (!done()) {
        if (timeout_us == 0) return TSQBX_PENDING;
        if (timeout_us < 0) S->cv.wait(lk, done);
        else if (!S->cv.wait_for(lk, std::chrono::microseconds(timeout_us), done)) return TSQBX_E_TIMEOUT;
    }
    const int st = r->status;
    S->requests.erase(it);
    return st;
}

int tsqbx_server_get_stats(tsqbx_server S, tsqbx_server_stats *st)
{
    if (!S || !st) return TSQBX_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> l = S->lat;
    std::sort(l.begin(), l.end());
    auto q = [&](double f) { return l.empty() ? 0.0 : 1e3 * l[(size_t)std::min<double>(l.size() - 1, std::floor(f * l.size()))]; };
    double mean = 0;
    for (double v : l) mean += v;
    st->p50_ms = q(0.50);
    st->p99_ms = q(0.99);
    st->mean_ms = l.empty() ? 0.0 : 1e3 * mean / l.size();
    st->max_ms = l.empty() ? 0.0 : 1e3 * l.back();
    st->completed = S->completed;
    st->failed = S->failed;
    st->rejected = S->rejected;
    st->queued = (int64_t)S->queue.size();
    st->running = (int64_t)S->running.size();
    st->plans_resident = (int64_t)S->plans.size();
    st->plans_created = S->created;
    st->plans_evicted = S->evicted;
    st->resident_bytes = S->resident;
    st->pair_terms_completed = S->pair_terms;
    st->span_s = S->any_done ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    st->merged = S->merged;
    return TSQBX_OK;
}

int tsqbx_server_reset_stats(tsqbx_server S)
{
    if (!S) return TSQBX_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat.clear();
    S->completed = S->failed = S->rejected = 0;
    S->pair_terms = 0;
    S->merged = 0;
    S->any_done = false;
    S->span_started = false;
    return TSQBX_OK;
}

int tsqbx_server_set_size_priority(tsqbx_server S, int on)
{
    if (!S) return TSQBX_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    S->size_priority = on != 0;
    return TSQBX_OK;
}

int tsqbx_server_set_laplace_fp64_path(tsqbx_server S, int precision)
{
    if (!S || (precision != TSQBX_FP64 && precision != TSQBX_DF64)) return TSQBX_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    S->laplace_fp64_as_df64 = precision == TSQBX_DF64;
    return TSQBX_OK;
}

int tsqbx_server_prepare(tsqbx_server S, int geom_id, const tsqbx_options *opt)
{
    if (!S || !opt) return TSQBX_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (geom_id < 0 || geom_id >= (int)S->geoms.size()) return TSQBX_E_INVAL;
    tsqbx_options o = *opt;
    if (S->size_priority) o.flags |= TSQBX_FLAG_SIZE_PRIORITY;
    if (S->laplace_fp64_as_df64 && o.kernel == TSQBX_LAPLACE && o.precision == TSQBX_FP64)
        o.precision = TSQBX_DF64;
    if (mergeable(o)) o.max_rhs = kServerMaxRhs;
    o.device = S->device;
    const PlanKey key{geom_id, (int)o.kernel, o.layers, (int)o.precision};
    auto it = S->plans.find(key);
    if (it != S->plans.end()) {
        it->second.last_use = ++S->use_clock;
        return TSQBX_OK;
    }
    const GeomCopy &g = *S->geoms[geom_id];
    const size_t need = estimate_bytes(g, o);
    if (need > S->budget) return TSQBX_E_NOMEM;
    if (S->resident + need > S->budget) S->evict_for(need);
    if (S->resident + need > S->budget) return TSQBX_E_BUSY;
    tsqbx_plan P = nullptr;
    const int rc = tsqbx_plan_create(&g.view, &o, &P);
    if (rc != TSQBX_OK) return rc;
    size_t bytes = 0;
    tsqbx_plan_footprint(P, &bytes);
    S->plans.emplace(key, PlanEntry{P, bytes, 0, ++S->use_clock});
    S->resident += bytes;
    ++S->created;
    return TSQBX_OK;
}

}  // extern "C"
