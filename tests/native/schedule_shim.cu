// schedule_shim.cu -- test-only C entry points into the plan's host-side work
// partition (csrc/schedule.cu, compiled into this shim unchanged), so that
// the CPU tests can check its invariants without a GPU.
#include "../../paper_1811_01110_gb300/csrc/schedule.cu"

extern "C" {

__attribute__((visibility("default"))) int shim_choose_lanes(int64_t nt, int64_t ns)
{
    return tsqbx::choose_lanes(nt, ns);
}

__attribute__((visibility("default"))) int shim_choose_lanes_weighted(int64_t nt, int64_t ns, double staging)
{
    return tsqbx::choose_lanes(nt, ns, staging);
}

__attribute__((visibility("default"))) double shim_staging_weight(int mixed)
{
    return mixed ? tsqbx::kStagingMixed : tsqbx::kStagingDefault;
}

__attribute__((visibility("default"))) int shim_priority_for_work(int64_t n_pairs, int kernel, int precision,
                                                                   int least, int greatest)
{
    return tsqbx::priority_for_work(n_pairs, kernel, precision, least, greatest);
}

__attribute__((visibility("default"))) int shim_cost_bucket(double cost) { return tsqbx::cost_bucket(cost); }

__attribute__((visibility("default"))) int shim_conventional_cheaper(int64_t nt, int64_t ns, int p,
                                                                      unsigned layers, int helmholtz)
{
    return tsqbx::conventional_cheaper(nt, ns, p, layers, helmholtz != 0) ? 1 : 0;
}

// The batch queue order: order[k] = index of the k-th item.
__attribute__((visibility("default"))) void shim_batch_queue_order(int64_t n, const int32_t *plan_of,
                                                                    const double *cost, int64_t *order)
{
    const std::vector<int64_t> o = tsqbx::batch_queue_order(std::vector<int32_t>(plan_of, plan_of + n),
                                                            std::vector<double>(cost, cost + n));
    for (int64_t i = 0; i < n; ++i) order[i] = o[(size_t)i];
}

// Items as 8 int32 each {group, slot_begin, n_tgt, L, src_lo, src_hi, part, pad}
// plus their costs; combine records as 4 int32 each {slot_begin, n_tgt, part, n_slices}.  With
// items == NULL only the counts are returned.
__attribute__((visibility("default"))) int shim_build_schedule(
    int64_t n_groups, const int64_t *q, const int64_t *slot_begin, const int64_t *nt, const int64_t *ns,
    int lanes_policy, int64_t max_iters, int n_sm, int64_t *n_items, int32_t *items, double *cost,
    int64_t *n_combine, int32_t *combine, int64_t *n_parts, int64_t *max_iters_used, double *utilisation)
{
    std::vector<tsqbx::GroupWork> groups((size_t)n_groups);
    for (int64_t i = 0; i < n_groups; ++i) groups[(size_t)i] = {q[i], slot_begin[i], nt[i], ns[i]};
    tsqbx::Schedule s;
    const int rc = tsqbx::build_schedule(groups, lanes_policy, max_iters, n_sm, s);
    if (rc != TSQBX_OK) return rc;
    *n_items = (int64_t)s.items.size();
    *n_combine = (int64_t)s.combine.size();
    *n_parts = s.n_parts;
    *max_iters_used = s.max_iters;
    *utilisation = s.lane_utilisation;
    if (!items) return rc;
    for (size_t i = 0; i < s.items.size(); ++i) {
        const tsqbx::Item &it = s.items[i].it;
        const int32_t v[8] = {it.group, it.slot_begin, it.n_tgt, it.L, it.src_lo, it.src_hi, it.part, it.pad};
        for (int k = 0; k < 8; ++k) items[8 * i + k] = v[k];
        cost[i] = s.items[i].cost;
    }
    for (size_t i = 0; i < s.combine.size(); ++i) {
        const tsqbx::Combine &c = s.combine[i];
        const int32_t v[4] = {c.slot_begin, c.n_tgt, c.part, c.n_slices};
        for (int k = 0; k < 4; ++k) combine[4 * i + k] = v[k];
    }
    return rc;
}

}  // extern "C"
