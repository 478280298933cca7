"""Serving runtime (tsqbx_server_*) and per-call order/wavenumber.

Continuous batching must not change results: every request's output equals
the output of evaluating it alone on a fresh plan (bit for bit: same plan
schedule, same kernels), within the stated tolerances of the oracle too."""
import ctypes
import time

import numpy as np
import pytest

import oracle
from helpers import cloud_geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01110_gb300 as pkg
    pkg.lib()
    return pkg


def _geoms():
    from tsqbx_inputs import configs
    rng = np.random.default_rng(71)
    g1 = cloud_geometry(rng, n_ctr=20, n_src=400, q_max=0.5, tgt_per_ctr=3, list_frac=0.6)
    g2, _ = configs.sphere(subdiv=2)
    g3, _, _ = configs.torus(24, 10)
    return [g1, g2, g3]


KINDS = [("laplace", ("slp", "dlp"), "fp64", 0.0), ("laplace", ("slp",), "mixed", 0.0),
         ("helmholtz", ("slp",), "fp64", 1.0), ("helmholtz", ("slp",), "fp64", 5.0)]


def test_plan_order_and_wavenumber_per_call(pkg):
    rng = np.random.default_rng(73)
    g = _geoms()[0]
    mu = rng.standard_normal(g.n_src)
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=5) as plan:
        for p in (0, 3, 9, 12):
            got = plan.eval(mu, p=p)
            with pkg.Plan(g, "laplace", ("slp", "dlp"), p=p) as ref_plan:
                ref = ref_plan.eval(mu)
            for l in ("slp", "dlp"):
                assert np.array_equal(got[l], ref[l])
    muc = mu + 0.3j * rng.standard_normal(g.n_src)
    with pkg.Plan(g, "helmholtz", ("slp",), p=4, k=2.0) as plan:
        for p, k in ((4, 2.0), (9, 7.5), (2, 0.5)):
            got = plan.eval(muc, p=p, k=k)["slp"]
            ref = oracle.tsqbx_helmholtz(g, p, k, muc)["slp"]
            assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-12


def test_results_same_alone_and_in_the_mix(pkg):
    geoms = _geoms()
    rng = np.random.default_rng(79)
    reqs = []
    with pkg.Server(hbm_budget=8 << 30, max_inflight=16) as srv:
        gids = [srv.add_geometry(g) for g in geoms]
        for i in range(40):
            gi = int(rng.integers(len(geoms)))
            kernel, layers, prec, k = KINDS[int(rng.integers(len(KINDS)))]
            p = int(rng.choice([3, 5, 9, 12]))
            g = geoms[gi]
            mu = rng.standard_normal(g.n_src)
            if kernel == "helmholtz":
                mu = mu + 1j * rng.standard_normal(g.n_src)
            rid, outs = srv.submit(gids[gi], mu, kernel, layers, p, k, prec)
            reqs.append((rid, outs, gi, kernel, layers, p, k, prec, mu))
        for rid, *_ in reqs:
            assert srv.poll(rid, timeout_us=-1)
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0 and st["rejected"] == 0
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
        assert st["plans_created"] <= len(geoms) * len(set((k[0], k[2]) for k in KINDS))
    tol = {"fp64": 1e-12, "mixed": 1e-6}
    for rid, outs, gi, kernel, layers, p, k, prec, mu in reqs:
        g = geoms[gi]
        with pkg.Plan(g, kernel, layers, p=p, k=k, precision=prec) as alone:
            ref = alone.eval(mu)
        for l in layers:
            assert np.array_equal(outs[l], ref[l]), (kernel, prec, p, l)
        if kernel == "laplace":
            ora = oracle.tsqbx_laplace(g, p, mu, slp="slp" in layers, dlp="dlp" in layers)
        else:
            ora = oracle.tsqbx_helmholtz(g, p, k, mu)
        for l in layers:
            assert np.max(np.abs(outs[l] - ora[l])) / np.max(np.abs(ora[l])) <= tol[prec]


def test_admission_eviction_and_rejection(pkg):
    geoms = _geoms()
    rng = np.random.default_rng(83)
    # a budget that holds the largest plan but never all three at once (the
    # server's Laplace single-layer plans hold scratch for four densities)
    fps = []
    for g in geoms[:3]:
        with pkg.Plan(g, "laplace", ("slp",), p=5, max_rhs=4) as probe:
            fps.append(probe.footprint())
    budget = max(fps) + min(fps) // 2
    assert budget < sum(fps)
    with pkg.Server(hbm_budget=budget, max_inflight=8) as srv:
        gids = [srv.add_geometry(g) for g in geoms]
        rids = []
        for i in range(12):
            gi = i % 3
            rid, _ = srv.submit(gids[gi], rng.standard_normal(geoms[gi].n_src), "laplace", ("slp",), 5)
            rids.append(rid)
        for rid in rids:
            assert srv.poll(rid, timeout_us=-1)
        st = srv.stats()
        assert st["completed"] == 12 and st["plans_evicted"] > 0
        assert st["resident_bytes"] <= budget
    # a plan that can never fit the budget is rejected, not queued forever
    with pkg.Server(hbm_budget=1 << 10, max_inflight=4) as srv:
        gid = srv.add_geometry(geoms[0])
        rid, _ = srv.submit(gid, np.ones(geoms[0].n_src), "laplace", ("slp",), 3)
        with pytest.raises(pkg.TsqbxError) as ei:
            srv.poll(rid, timeout_us=-1)
        assert ei.value.code == -3


def test_poll_timeout(pkg):
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus(64, 24)
    with pkg.Server() as srv:
        gid = srv.add_geometry(g)
        rid, _ = srv.submit(gid, mu, "laplace", ("slp", "dlp"), 9)
        rc = pkg.lib().tsqbx_server_poll(srv._h, ctypes.c_uint64(rid), 1)
        assert rc in (-5, 1, 0)          # timed out (plan creation alone takes ms), or done
        t0 = time.perf_counter()
        assert srv.poll(rid, timeout_us=-1)
        assert time.perf_counter() - t0 < 60
        assert pkg.lib().tsqbx_server_poll(srv._h, ctypes.c_uint64(rid), 0) == -7   # retired


def test_size_priority_leaves_results_unchanged(pkg):
    """TSQBX_FLAG_SIZE_PRIORITY only changes the streams' priority: the same
    plan with and without it gives bit-identical results."""
    g = _geoms()[1]
    mu = np.random.default_rng(5).standard_normal(g.n_src)
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=9) as a, \
            pkg.Plan(g, "laplace", ("slp", "dlp"), p=9, size_priority=True) as b:
        ra, rb = a.eval(mu), b.eval(mu)
    for layer in ("slp", "dlp"):
        assert np.array_equal(ra[layer], rb[layer])


def test_size_priority_server_matches_fifo_server(pkg):
    """The server's size-priority policy changes only the order in which
    concurrent work is dispatched: every request's result equals the FIFO
    server's bit for bit."""
    geoms = _geoms()
    rng = np.random.default_rng(19)
    reqs = [(i % 3, rng.standard_normal(geoms[i % 3].n_src)) for i in range(9)]
    results = []
    for prio in (False, True):
        with pkg.Server(hbm_budget=4 << 30, max_inflight=8, size_priority=prio) as srv:
            gids = [srv.add_geometry(g) for g in geoms]
            subs = [srv.submit(gids[gi], mu, "laplace", ("slp", "dlp"), 7) for gi, mu in reqs]
            for rid, _ in subs:
                assert srv.poll(rid, timeout_us=-1)
            results.append([outs for _, outs in subs])
    for a, b in zip(*results):
        for layer in ("slp", "dlp"):
            assert np.array_equal(a[layer], b[layer])


def test_laplace_fp64_requests_on_the_double_float_path(pkg):
    """With the server's Laplace FP64 path set to double-float, FP64 requests
    run on DF64 plans: bit-identical to a DF64 plan evaluated alone, within
    the FP64 bar (1e-12) of the oracle; mixed and Helmholtz requests are
    unaffected."""
    geoms = _geoms()
    rng = np.random.default_rng(89)
    reqs = []
    with pkg.Server(hbm_budget=8 << 30, max_inflight=8, laplace_fp64_path="df64") as srv:
        gids = [srv.add_geometry(g) for g in geoms]
        for i in range(12):
            gi = i % len(geoms)
            kernel, layers, prec, k = KINDS[i % len(KINDS)]
            g = geoms[gi]
            mu = rng.standard_normal(g.n_src)
            if kernel == "helmholtz":
                mu = mu + 1j * rng.standard_normal(g.n_src)
            rid, outs = srv.submit(gids[gi], mu, kernel, layers, 9, k, prec)
            reqs.append((rid, outs, gi, kernel, layers, k, prec, mu))
        for rid, *_ in reqs:
            assert srv.poll(rid, timeout_us=-1)
    for rid, outs, gi, kernel, layers, k, prec, mu in reqs:
        g = geoms[gi]
        run_as = "df64" if (kernel == "laplace" and prec == "fp64") else prec
        with pkg.Plan(g, kernel, layers, p=9, k=k, precision=run_as) as alone:
            ref = alone.eval(mu)
        for l in layers:
            assert np.array_equal(outs[l], ref[l]), (kernel, prec, l)
        if kernel == "laplace" and prec == "fp64":
            ora = oracle.tsqbx_laplace(g, 9, mu, slp=True, dlp="dlp" in layers)
            for l in layers:
                assert np.max(np.abs(outs[l] - ora[l])) / np.max(np.abs(ora[l])) <= 1e-12
