"""Autotuner and schedule controls (tsqbx_plan_autotune / set / get tuning)."""
import numpy as np
import pytest

import oracle
from helpers import cloud_geometry

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01110_gb300 as pkg
    pkg.lib()
    return torch, pkg


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_autotune_keeps_results_and_caches(env, precision, tol):
    torch, pkg = env
    rng = np.random.default_rng(41)
    g = cloud_geometry(rng, n_ctr=30, n_src=600, q_max=0.5, tgt_per_ctr=9, list_frac=0.6)
    mu = rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_laplace(g, 7, mu, slp=True, dlp=True)
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=7, precision=precision) as plan:
        t = plan.autotune(torch.from_numpy(mu).cuda(), repeats=3)
        assert t["max_item_iters"] in (64, 128, 256, 512, 1024, 2048) or t["max_item_iters"] > 0
        assert t["lanes_per_target"] in (0, 1, 2, 4, 8, 16)
        assert t["tile_depth"] in (32, 64, 128)
        assert t["p_unroll"] in (0, 1, 2, 4)
        assert t["kernel_ms"] > 0
        assert plan.get_tuning()["max_item_iters"] == t["max_item_iters"]
        assert plan.get_tuning()["tile_depth"] == t["tile_depth"]
        out = plan.eval(mu)
        for l in ("slp", "dlp"):
            assert relerr(out[l], ref[l]) <= tol
    # a new plan with the same shape starts from the cached choice
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=7, precision=precision, use_tuned=True) as plan2:
        assert plan2.get_tuning() == {"lanes_per_target": t["lanes_per_target"],
                                      "max_item_iters": t["max_item_iters"], "tile_depth": t["tile_depth"],
                                      "p_unroll": t["p_unroll"], "fp64_share": t["fp64_share"]}


def test_set_tuning_roundtrip(env):
    torch, pkg = env
    rng = np.random.default_rng(43)
    g = cloud_geometry(rng, n_ctr=10, n_src=300, tgt_per_ctr=5)
    mu = rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_laplace(g, 5, mu)["slp"]
    with pkg.Plan(g, "laplace", ("slp",), p=5) as plan:
        for lanes, iters, depth, unroll in ((1, 3, 32, 0), (4, 50, 128, 2), (0, 1, 0, 1), (32, 1000, 64, 4)):
            plan.set_tuning(lanes, iters, depth, unroll)
            assert plan.get_tuning() == {"lanes_per_target": lanes, "max_item_iters": iters,
                                         "tile_depth": depth or 64, "p_unroll": unroll, "fp64_share": 0}
            assert relerr(plan.eval(mu)["slp"], ref) <= 1e-12
        info = plan.info()
        assert info["launches_per_eval"] in (2, 3)


@pytest.mark.parametrize("depth", [32, 64, 128])
@pytest.mark.parametrize("kernel,precision,tol", [("laplace", "fp64", 1e-12), ("laplace", "mixed", 1e-6),
                                                  ("laplace", "df64", 1e-12), ("helmholtz", "fp64", 1e-12)])
def test_every_tile_depth_matches_the_oracle(env, depth, kernel, precision, tol):
    """Each staging depth (sources per shared-memory tile) over lists that are
    not multiples of it (ragged last tiles), several lane counts per target,
    and every layer, against the oracle."""
    torch, pkg = env
    rng = np.random.default_rng(47 + depth)
    g = cloud_geometry(rng, n_ctr=8, n_src=700, q_max=0.5, tgt_per_ctr=11, list_frac=0.43)
    layers = ("slp", "dlp", "sp")
    if kernel == "helmholtz":
        mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
        ref = oracle.tsqbx_helmholtz(g, 8, 3.0, mu, slp=True, dlp=True, sp=True)
        kw = {"k": 3.0}
    else:
        mu = rng.standard_normal(g.n_src)
        ref = oracle.tsqbx_laplace(g, 8, mu, slp=True, dlp=True, sp=True)
        kw = {"precision": precision}
    for lanes in (0, 3, 8):
        with pkg.Plan(g, kernel, layers, p=8, tile_depth=depth, lanes_per_target=lanes, **kw) as plan:
            assert plan.get_tuning()["tile_depth"] == depth
            out = plan.eval(mu)
        for l in layers:
            assert relerr(out[l], ref[l]) <= tol, (l, lanes, relerr(out[l], ref[l]))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("layers", [("slp",), ("slp", "dlp"), ("slp", "dlp", "sp")])
@pytest.mark.parametrize("unroll", [1, 2, 4])
def test_runtime_order_kernels_match_the_oracle(env, precision, tol, layers, unroll):
    """The runtime-order kernels (p_unroll 1, 2, 4: one kernel for every
    order, the loop over n unrolled by that factor, coefficients from
    constant memory) against the oracle at every order 0..20 of one plan
    (per-call orders), sliced lists and several lane counts, and against the
    per-order kernels to rounding."""
    torch, pkg = env
    rng = np.random.default_rng(53 + unroll)
    g = cloud_geometry(rng, n_ctr=10, n_src=260, q_max=0.6, tgt_per_ctr=4, list_frac=0.7)
    mu = rng.standard_normal(g.n_src)
    kw = dict(slp="slp" in layers, dlp="dlp" in layers, sp="sp" in layers)
    with pkg.Plan(g, "laplace", layers, p=9, precision=precision, p_unroll=unroll, max_item_iters=3,
                  lanes_per_target=3) as rt, \
            pkg.Plan(g, "laplace", layers, p=9, precision=precision, max_item_iters=3,
                     lanes_per_target=3) as fixed:
        assert rt.get_tuning()["p_unroll"] == unroll
        for p in range(0, 21):
            ref = oracle.tsqbx_laplace(g, p, mu, **kw)
            a, b = rt.eval(mu, p=p), fixed.eval(mu, p=p)
            for l in layers:
                if not np.any(ref[l]):                 # S' at p = 0 vanishes
                    assert not np.any(a[l]) and not np.any(b[l]), (p, l)
                    continue
                assert relerr(a[l], ref[l]) <= tol, (p, l)
                assert relerr(a[l], b[l]) <= (1e-14 if precision == "fp64" else 2e-6), (p, l)


def test_autotune_searches_the_order_loop_forms(env):
    torch, pkg = env
    rng = np.random.default_rng(59)
    g = cloud_geometry(rng, n_ctr=30, n_src=600, q_max=0.5, tgt_per_ctr=9, list_frac=0.6)
    mu = rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_laplace(g, 14, mu, slp=True, dlp=True)
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=14, precision="fp64") as plan:
        t = plan.autotune(torch.from_numpy(mu).cuda(), repeats=2)
        assert t["p_unroll"] in (0, 1, 2, 4) and plan.get_tuning()["p_unroll"] == t["p_unroll"]
        out = plan.eval(mu)
        for l in ("slp", "dlp"):
            assert relerr(out[l], ref[l]) <= 1e-12
    with pkg.Plan(g, "helmholtz", ("slp",), p=6, k=2.0) as plan:     # no runtime-order form here
        assert plan.autotune(torch.from_numpy(mu + 0j).cuda(), repeats=1)["p_unroll"] == 0
        with pytest.raises(pkg.TsqbxError) as e:
            plan.set_tuning(0, 0, 0, 2)
        assert e.value.code == -9


@pytest.mark.parametrize("layers", [("slp",), ("slp", "dlp"), ("slp", "dlp", "sp")])
@pytest.mark.parametrize("share", [1, 5, 10, 20])
def test_double_float_plans_with_fp64_items(env, layers, share):
    """Double-float plans whose items with (index mod 20) < fp64_share run
    the native FP64 body in the same launch: every order 0..20 against the
    oracle at the FP64 bar, sliced lists, several lane counts; each result
    the same from run to run."""
    torch, pkg = env
    rng = np.random.default_rng(61 + share)
    g = cloud_geometry(rng, n_ctr=16, n_src=300, q_max=0.6, tgt_per_ctr=4, list_frac=0.7)
    mu = rng.standard_normal(g.n_src)
    kw = dict(slp="slp" in layers, dlp="dlp" in layers, sp="sp" in layers)
    with pkg.Plan(g, "laplace", layers, p=9, precision="df64", fp64_share=share, max_item_iters=3,
                  lanes_per_target=3) as plan:
        assert plan.get_tuning()["fp64_share"] == share
        assert plan.info()["n_items"] >= 20
        for p in range(0, 21):
            ref = oracle.tsqbx_laplace(g, p, mu, **kw)
            a = plan.eval(mu, p=p)
            for l in layers:
                if not np.any(ref[l]):
                    assert not np.any(a[l]), (p, l)
                    continue
                assert relerr(a[l], ref[l]) <= 1e-12, (p, l)
        b = plan.eval(mu, p=20)
        for l in layers:
            assert np.array_equal(a[l], b[l])


def test_fp64_share_tuning_and_rejection(env):
    torch, pkg = env
    rng = np.random.default_rng(67)
    g = cloud_geometry(rng, n_ctr=30, n_src=600, q_max=0.5, tgt_per_ctr=9, list_frac=0.6)
    mu = rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_laplace(g, 9, mu, slp=True, dlp=True)
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=9, precision="df64") as plan:
        t = plan.autotune(torch.from_numpy(mu).cuda(), repeats=2)
        assert t["fp64_share"] in (0, 1, 2, 3) and t["p_unroll"] == 0
        out = plan.eval(mu)
        for l in ("slp", "dlp"):
            assert relerr(out[l], ref[l]) <= 1e-12
        plan.set_tuning(0, 0, 0, 0, 7)
        assert plan.get_tuning()["fp64_share"] == 7
    with pkg.Plan(g, "laplace", ("slp",), p=9, precision="mixed") as plan:
        with pytest.raises(pkg.TsqbxError) as e:
            plan.set_tuning(0, 0, 0, 0, 2)
        assert e.value.code == -9
