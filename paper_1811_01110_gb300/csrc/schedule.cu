// schedule.cu -- host-side work partition of a plan: warp items, lanes per
// target, source slices and their combine records, the queue order, and the
// cost model that sends centers to the conventional path.  Pure host code
// (no CUDA calls), so it can be built and checked without a GPU.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <vector>

#include "plan_internal.h"

namespace tsqbx {

int cost_bucket(double cost) { return cost > 0 ? (int)std::floor(2.0 * std::log2(cost)) : -1; }

// Cost per unit in ns, measured on GB300 (torus 96 x 36, every center on one
// path, kernel time of whole evaluations; orders 2..20 for Laplace, 2..12 for
// Helmholtz k = 10, whose target-specific sums are Clenshaw's) and fitted in
// q = p + 1, the form of Table 2:
//   target-specific, per (target, source) pair:      ts0 + ts1 q
//   P2QBXL, per (center, source):                    c0 + c1 q + c2 q^2
//   QBXL2P, per warp item (a center's <= 32 targets): w0 + w1 q + w2 q^2
// Indexed by the layer bits (SLP 1, DLP 2, S' 4); S' alone costs as SLP + S'.
struct ConvCostFit {
    double ts[2], p2l[3], l2p[3];
};
constexpr ConvCostFit kLaplaceCost[8] = {
    {{0, 0}, {0, 0, 0}, {0, 0, 0}},
    {{0.02604, 0.005689}, {0.1122, -0.02055, 0.007475}, {0.1807, -0.2473, 0.2366}},     // slp
    {{0.0534, 0.007602}, {0.1749, -0.04791, 0.01721}, {0.2934, -0.3058, 0.2418}},       // dlp
    {{0.05343, 0.007597}, {0.0906, -0.01624, 0.01806}, {-0.13, -0.1184, 0.3189}},       // slp+dlp
    {{0.04471, 0.007716}, {0.1123, -0.02061, 0.007484}, {-1.655, 0.2953, 0.5637}},      // sp
    {{0.04471, 0.007716}, {0.1123, -0.02061, 0.007484}, {-1.655, 0.2953, 0.5637}},      // slp+sp
    {{0.06253, 0.007715}, {0.09266, -0.01707, 0.01811}, {-1.418, 0.1222, 0.675}},       // dlp+sp
    {{0.06249, 0.007722}, {0.09095, -0.01642, 0.01806}, {-0.8973, -0.09392, 0.6941}},   // slp+dlp+sp
};
constexpr ConvCostFit kHelmholtzCost[8] = {
    {{0, 0}, {0, 0, 0}, {0, 0, 0}},
    {{0.09568, 0.009309}, {0.08981, 0.01622, 0.01129}, {9.758, 2.279, 0.2306}},  // slp
    {{0.1096, 0.02873}, {0.1014, 0.03242, 0.02055}, {10.16, 2.145, 0.2431}},     // dlp
    {{0.1096, 0.02874}, {0.1264, 0.03291, 0.02829}, {10.99, 1.983, 0.4262}},     // slp+dlp
    {{0.1106, 0.02201}, {0.08737, 0.01723, 0.01122}, {11.05, 2.606, 0.7122}},    // sp
    {{0.1106, 0.02201}, {0.08737, 0.01723, 0.01122}, {11.05, 2.606, 0.7122}},    // slp+sp
    {{0.1388, 0.03545}, {0.1284, 0.03217, 0.02833}, {10.61, 2.948, 0.8605}},     // dlp+sp
    {{0.1389, 0.03545}, {0.1285, 0.0325, 0.02831}, {10.79, 2.812, 0.872}},       // slp+dlp+sp
};

bool conventional_cheaper(int64_t nt, int64_t ns, int p, unsigned layers, bool helmholtz)
{
    const ConvCostFit &f = (helmholtz ? kHelmholtzCost : kLaplaceCost)[layers & 7u];
    const double q = p + 1.0;
    const double ts = f.ts[0] + f.ts[1] * q;
    const double p2l = f.p2l[0] + q * (f.p2l[1] + q * f.p2l[2]);
    const double l2p = f.l2p[0] + q * (f.l2p[1] + q * f.l2p[2]);
    const double warps = (double)((nt + 31) / 32);
    return (double)ns * p2l + warps * l2p < (double)nt * (double)ns * ts;
}

int priority_for_work(int64_t n_pairs, int kernel, int precision, int least, int greatest)
{
    const double cost = kernel == TSQBX_HELMHOLTZ ? 4.0
                        : precision == TSQBX_MIXED ? 0.03
                        : precision == TSQBX_DF64  ? 0.25
                                                   : 1.0;
    const double work = std::max(1.0, (double)n_pairs * cost);
    const int level = std::min(std::max((int)std::floor(std::log10(work)) - 5, 0), least - greatest);
    return greatest + level;
}

int choose_lanes(int64_t nt, int64_t ns, double staging)
{
    int best = 1;
    double best_cost = 1e300;
    for (int L = 1; L <= 32; ++L) {
        const int64_t tpw = 32 / L;
        const int64_t items = (nt + tpw - 1) / tpw;
        const double cost = (double)items * ((double)((ns + L - 1) / L) + staging * (double)ns / 32.0 + 4.0);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = L; }
    }
    return best;
}

int build_schedule(const std::vector<GroupWork> &groups, int lanes_policy, int64_t max_iters,
                   int n_sm, Schedule &out, double staging)
{
    struct Chunk { int64_t q, slot, m; int L; int64_t ns; };
    std::vector<Chunk> chunks;
    int64_t total_iters = 0;
    for (const GroupWork &w : groups) {
        const int L = lanes_policy ? lanes_policy : choose_lanes(w.nt, w.ns, staging);
        const int64_t tpw = 32 / L;
        for (int64_t b = 0; b < w.nt; b += tpw) {
            chunks.push_back({w.q, w.slot_begin + b, std::min(tpw, w.nt - b), L, w.ns});
            total_iters += (w.ns + L - 1) / L;
        }
    }
    if (max_iters <= 0)
        max_iters = std::min<int64_t>(512, std::max<int64_t>(32, total_iters / ((int64_t)n_sm * 48)));
    Schedule s;
    s.lanes_policy = lanes_policy;
    s.max_iters = max_iters;
    double used = 0.0, offered = 0.0;
    for (const Chunk &c : chunks) {
        const int64_t iters = (c.ns + c.L - 1) / c.L;
        const int64_t K = iters > max_iters ? (iters + max_iters - 1) / max_iters : 1;
        int64_t base = -1;
        if (K > 1) {
            base = s.n_parts;
            s.n_parts += K * c.m;
            if (s.n_parts > INT32_MAX) return TSQBX_E_INVAL;
            s.combine.push_back({(int32_t)c.slot, (int32_t)c.m, (int32_t)base, (int32_t)K});
        }
        for (int64_t k = 0; k < K; ++k) {
            const int64_t lo = c.ns * k / K, hi = c.ns * (k + 1) / K;
            const double cost = (double)((hi - lo + c.L - 1) / c.L) + 0.25 * (double)(hi - lo) / 32.0 + 4.0;
            Item it;
            it.group = (int32_t)c.q;
            it.slot_begin = (int32_t)c.slot;
            it.n_tgt = (int32_t)c.m;
            it.L = c.L;
            it.src_lo = (int32_t)lo;
            it.src_hi = (int32_t)hi;
            it.part = K > 1 ? (int32_t)(base + k * c.m) : -1;
            it.pad = 0;
            s.items.push_back({it, cost});
            used += cost * (double)(c.m * c.L);
            offered += cost * 32.0;
        }
    }
    // heaviest first, by half-octave cost bucket; within a bucket the items
    // keep list order, so neighbouring groups (which share many sources) run
    // close together in time and share cached source data
    std::stable_sort(s.items.begin(), s.items.end(), [](const Schedule::Entry &a, const Schedule::Entry &b) {
        return cost_bucket(a.cost) > cost_bucket(b.cost);
    });
    s.lane_utilisation = offered > 0 ? used / offered : 1.0;
    out = std::move(s);
    return TSQBX_OK;
}

std::vector<int64_t> batch_queue_order(const std::vector<int32_t> &plan_of, const std::vector<double> &cost)
{
    // plans with more work first (ties: the lower index), then each plan's
    // items in their own schedule order: heaviest half-octave bucket first
    int32_t n_plans = 0;
    for (int32_t q : plan_of) n_plans = std::max(n_plans, q + 1);
    std::vector<double> work((size_t)n_plans, 0.0);
    for (size_t i = 0; i < plan_of.size(); ++i) work[(size_t)plan_of[i]] += cost[i];
    std::vector<int32_t> rank((size_t)n_plans);
    {
        std::vector<int32_t> byw((size_t)n_plans);
        for (int32_t q = 0; q < n_plans; ++q) byw[(size_t)q] = q;
        std::stable_sort(byw.begin(), byw.end(), [&](int32_t a, int32_t b) { return work[(size_t)a] > work[(size_t)b]; });
        for (int32_t r = 0; r < n_plans; ++r) rank[(size_t)byw[(size_t)r]] = r;
    }
    std::vector<int64_t> order(plan_of.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int64_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const int32_t ra = rank[(size_t)plan_of[(size_t)a]], rb = rank[(size_t)plan_of[(size_t)b]];
        if (ra != rb) return ra < rb;
        return cost_bucket(cost[(size_t)a]) > cost_bucket(cost[(size_t)b]);
    });
    return order;
}

}  // namespace tsqbx
