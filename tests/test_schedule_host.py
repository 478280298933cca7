"""The plan's host-side work partition (csrc/schedule.cu), built alone into a
test shim and checked without a GPU:

* every (target, listed source) pair of every group falls in exactly one warp
  item, and targets with empty lists still get one item (which writes 0);
* an item holds at most 32/L targets of one group, with 1 <= L <= 32, and no
  lane runs more than the iteration cap;
* sliced lists get one combine record each, whose partial blocks are disjoint
  and cover [0, n_parts);
* the queue runs in half-octave cost buckets, heaviest first, keeping list
  order within a bucket; a persistent batch's queue runs plan by plan;
* the size-priority levels: one per decade of work above 1e5 Laplace-FP64
  pair equivalents, smallest plans highest, clamped to the device's range;
* the cost model's choice between the target-specific and the conventional
  path matches the measured faster path on the torus 96 x 36 cases
  (1/4/16/64 targets per center; Laplace SLP+DLP p = 9, Helmholtz SLP+DLP
  k = 10 p = 12).
"""
import ctypes
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

i64p = ctypes.POINTER(ctypes.c_int64)
i32p = ctypes.POINTER(ctypes.c_int32)
f64p = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def shim():
    from helpers import native_shim
    path = native_shim("schedule_shim")
    if path is None:
        pytest.skip("no nvcc")
    L = ctypes.CDLL(path)
    L.shim_build_schedule.argtypes = [ctypes.c_int64, i64p, i64p, i64p, i64p, ctypes.c_int, ctypes.c_int64,
                                      ctypes.c_int, i64p, i32p, f64p, i64p, i32p, i64p, i64p, f64p]
    L.shim_choose_lanes.argtypes = [ctypes.c_int64, ctypes.c_int64]
    L.shim_choose_lanes_weighted.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double]
    L.shim_staging_weight.argtypes = [ctypes.c_int]
    L.shim_staging_weight.restype = ctypes.c_double
    L.shim_cost_bucket.argtypes = [ctypes.c_double]
    L.shim_priority_for_work.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.shim_conventional_cheaper.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint,
                                            ctypes.c_int]
    return L


def schedule(L, nt, ns, lanes=0, max_iters=0, n_sm=152):
    nt = np.asarray(nt, np.int64)
    ns = np.asarray(ns, np.int64)
    q = np.arange(len(nt), dtype=np.int64)
    slot = np.concatenate([[0], np.cumsum(nt)[:-1]]).astype(np.int64)
    n_items, n_comb, n_parts, mi = (ctypes.c_int64() for _ in range(4))
    util = ctypes.c_double()
    args = [len(nt), q.ctypes.data_as(i64p), slot.ctypes.data_as(i64p), nt.ctypes.data_as(i64p),
            ns.ctypes.data_as(i64p), lanes, max_iters, n_sm]
    rc = L.shim_build_schedule(*args, ctypes.byref(n_items), None, None, ctypes.byref(n_comb), None,
                               ctypes.byref(n_parts), ctypes.byref(mi), ctypes.byref(util))
    if rc != 0:
        return rc, None
    items = np.zeros((max(n_items.value, 1), 8), np.int32)
    cost = np.zeros(max(n_items.value, 1))
    comb = np.zeros((max(n_comb.value, 1), 4), np.int32)
    rc = L.shim_build_schedule(*args, ctypes.byref(n_items), items.ctypes.data_as(i32p), cost.ctypes.data_as(f64p),
                               ctypes.byref(n_comb), comb.ctypes.data_as(i32p), ctypes.byref(n_parts),
                               ctypes.byref(mi), ctypes.byref(util))
    assert rc == 0
    return rc, dict(items=items[:n_items.value], cost=cost[:n_items.value], comb=comb[:n_comb.value],
                    n_parts=n_parts.value, max_iters=mi.value, util=util.value, nt=nt, ns=ns, slot=slot)


def check_partition(L, s):
    items, nt, ns, slot = s["items"], s["nt"], s["ns"], s["slot"]
    # coverage: per target, the source ranges of its items tile [0, ns) exactly once
    per_target = {}
    for g_, sb, m, Ln, lo, hi, part, pad in items:
        assert 1 <= Ln <= 32 and 1 <= m <= 32 // Ln, (m, Ln)
        assert slot[g_] <= sb and sb + m <= slot[g_] + nt[g_]
        assert 0 <= lo <= hi <= ns[g_]
        assert -(-(hi - lo) // Ln) <= s["max_iters"], (hi - lo, Ln, s["max_iters"])
        for t in range(sb, sb + m):
            per_target.setdefault(t, []).append((lo, hi))
    for gi in range(len(nt)):
        for t in range(slot[gi], slot[gi] + nt[gi]):
            r = sorted(per_target.get(int(t), []))
            assert r, ("target without an item", t)
            assert r[0][0] == 0 and r[-1][1] == ns[gi]
            assert all(a[1] == b[0] for a, b in zip(r, r[1:])), r
            assert sum(1 for x in r if x[1] > x[0]) == len(r) or ns[gi] == 0
    assert sum(len(v) for v in per_target.values()) == int(items[:, 2].sum())
    # slices and their combine records
    used = np.zeros(max(s["n_parts"], 1), np.int64)
    by_base = {}
    for g_, sb, m, Ln, lo, hi, part, pad in items:
        if part >= 0:
            used[part:part + m] += 1
    assert s["n_parts"] == 0 or np.all(used[:s["n_parts"]] == 1)
    for sb, m, base, K in s["comb"]:
        assert K > 1
        by_base[int(base)] = (int(sb), int(m), int(K))
    sliced = items[items[:, 6] >= 0]
    for sb, m, base_k in zip(sliced[:, 1], sliced[:, 2], sliced[:, 6]):
        owner = max(b for b in by_base if b <= base_k)
        osb, om, oK = by_base[owner]
        assert osb == sb and om == m and (base_k - owner) % m == 0 and (base_k - owner) // m < oK
    assert sum(m * K for _, m, _, K in s["comb"]) == s["n_parts"]
    # queue order: cost buckets non-increasing; list order kept within a bucket
    buckets = np.array([L.shim_cost_bucket(c) for c in s["cost"]])
    assert np.all(np.diff(buckets) <= 0)
    for b in np.unique(buckets):
        sel = items[buckets == b]
        keys = list(zip(sel[:, 0], sel[:, 1], sel[:, 4]))
        assert keys == sorted(keys)
    assert 0.0 < s["util"] <= 1.0 + 1e-12


CASES = [
    ("uniform", [4] * 50, [650] * 50),
    ("ragged", [1, 2, 5, 31, 32, 33, 100, 7], [0, 1, 63, 64, 65, 1000, 30000, 5]),
    ("empty lists", [3, 1, 40], [0, 0, 0]),
    ("empty groups", [0, 5, 0, 2], [100, 200, 300, 0]),
    ("one long list", [1], [200000]),
]


@pytest.mark.parametrize("name,nt,ns", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("lanes", [0, 1, 2, 8, 32])
@pytest.mark.parametrize("max_iters", [0, 1, 7, 512])
def test_items_partition_every_pair_once(shim, name, nt, ns, lanes, max_iters):
    rc, s = schedule(shim, nt, ns, lanes, max_iters)
    assert rc == 0
    if max_iters > 0:
        assert s["max_iters"] == max_iters
    else:
        assert 32 <= s["max_iters"] <= 512
    check_partition(shim, s)


def test_random_group_mixes(shim):
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(1, 60))
        nt = rng.integers(0, 70, n)
        ns = np.where(rng.uniform(size=n) < 0.1, 0, np.exp(rng.uniform(0, 9, n)).astype(np.int64))
        rc, s = schedule(shim, nt, ns, int(rng.choice([0, 1, 4, 16])), int(rng.choice([0, 3, 64])))
        assert rc == 0
        check_partition(shim, s)


def test_slice_count_overflow_is_rejected(shim):
    # 32 targets x 2^27 slices of one source each would need 2^32 partial blocks
    rc, _ = schedule(shim, [32], [2 ** 27], lanes=1, max_iters=1)
    assert rc == -1


def test_lane_choice_extremes(shim):
    assert shim.shim_choose_lanes(1, 100000) == 32          # one target, long list: the whole warp
    assert shim.shim_choose_lanes(64, 1) == 1               # many targets, one source: one lane each
    for nt, ns in ((4, 650), (16, 650), (1, 50), (100, 100000)):
        L = shim.shim_choose_lanes(nt, ns)
        assert 1 <= L <= 32


def test_lane_choice_staging_weight(shim):
    """Staging weighs more for the mixed plans (their per-pair arithmetic is
    cheap) than for FP64 and df64; a heavier staging weight never picks more
    lanes per target (fewer lanes: more targets share a staged tile), and the
    default weight is the unweighted call's."""
    assert shim.shim_staging_weight(1) > shim.shim_staging_weight(0) > 0
    w0 = shim.shim_staging_weight(0)
    for nt, ns in ((4, 650), (10, 456), (21, 547), (53, 318), (7, 29475), (1, 195)):
        assert shim.shim_choose_lanes_weighted(nt, ns, w0) == shim.shim_choose_lanes(nt, ns)
        Ls = [shim.shim_choose_lanes_weighted(nt, ns, w) for w in (0.0, 0.25, 0.5, 1.0, 4.0)]
        assert all(a >= b for a, b in zip(Ls, Ls[1:])), (nt, ns, Ls)
    # a single target keeps the whole warp whatever the weight
    assert shim.shim_choose_lanes_weighted(1, 5000, 4.0) == 32


@pytest.mark.parametrize("helmholtz,p", [(0, 9), (1, 12)])
def test_cost_model_picks_the_measured_faster_path(shim, helmholtz, p):
    """Torus 96 x 36 (about 650 listed sources per center), SLP+DLP: the
    target-specific path was faster at 1 and 4 targets per center, the
    conventional path at 16 and 64, for both kernels."""
    layers = 3
    for nt, conv_faster in ((1, False), (4, False), (16, True), (64, True)):
        assert shim.shim_conventional_cheaper(nt, 650, p, layers, helmholtz) == int(conv_faster), nt
    # more targets per center never turn the choice back
    picks = [shim.shim_conventional_cheaper(nt, 650, p, layers, helmholtz) for nt in range(1, 200)]
    assert picks == sorted(picks)


def test_size_priority_levels(shim):
    """Priority range as CUDA reports it: greatest (highest priority) is the
    numerically smaller value, e.g. [-5, 0]."""
    least, greatest = 0, -5
    lap, helm = 0, 1
    fp64, mixed, df64 = 0, 1, 2
    f = lambda n, k=lap, pr=fp64: shim.shim_priority_for_work(n, k, pr, least, greatest)
    assert f(0) == greatest and f(10 ** 5) == greatest and f(999_999) == greatest
    assert f(10 ** 6) == greatest + 1 and f(10 ** 8) == greatest + 3
    assert f(10 ** 12) == least                                   # clamped to the lowest priority
    levels = [f(int(10 ** e)) for e in np.arange(0, 13, 0.5)]
    assert levels == sorted(levels)                               # more work, never a higher priority
    # per-pair costs: Helmholtz 4x, mixed 0.03x, df64 0.25x of Laplace FP64
    assert f(2_500_000, helm) == f(10 ** 7)
    assert f(10 ** 8, lap, mixed) == f(3 * 10 ** 6)
    assert f(4 * 10 ** 6, lap, df64) == f(10 ** 6)
    # a device with a single priority puts everything at it
    assert shim.shim_priority_for_work(10 ** 9, lap, fp64, 0, 0) == 0


def test_batch_queue_runs_plan_by_plan(shim):
    """A persistent batch's queue: every item exactly once, the items of one
    plan contiguous, the plans in decreasing total work, and each plan's items
    in decreasing half-octave cost bucket, keeping their own order within a
    bucket (a surface's sources stay in L2 while its items run)."""
    L = shim
    L.shim_batch_queue_order.argtypes = [ctypes.c_int64, i32p, f64p, i64p]
    rng = np.random.default_rng(3)
    n = 5000
    plan_of = rng.integers(0, 13, n).astype(np.int32)
    cost = rng.lognormal(3.0, 1.2, n)
    order = np.zeros(n, np.int64)
    L.shim_batch_queue_order(n, plan_of.ctypes.data_as(i32p), cost.ctypes.data_as(f64p), order.ctypes.data_as(i64p))
    assert np.array_equal(np.sort(order), np.arange(n))
    plans = plan_of[order]
    runs = [plans[0]] + [b for a, b in zip(plans[:-1], plans[1:]) if a != b]
    assert len(runs) == len(set(runs))                       # contiguous per plan
    work = {q: cost[plan_of == q].sum() for q in set(runs)}
    assert all(work[a] >= work[b] for a, b in zip(runs[:-1], runs[1:]))
    bucket = lambda c: int(np.floor(2.0 * np.log2(c)))
    for q in runs:
        mine = order[plans == q]
        b = [bucket(c) for c in cost[mine]]
        assert all(x >= y for x, y in zip(b[:-1], b[1:]))
        for k in set(b):                                     # stable within a bucket
            same = mine[np.array(b) == k]
            assert np.all(np.diff(same) > 0)
