"""GPU parity: libtsqbx (through the C ABI) against the FP64 CPU oracle.

Tolerances (max-norm relative: max_t |u_gpu - u_oracle| / max_t |u_oracle|,
per output layer):  FP64 mode 1e-12,  mixed mode 1e-6.
"""
import numpy as np
import pytest

import oracle
from helpers import cloud_geometry
from tsqbx_inputs import configs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6, "df64": 1e-12}


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01110_gb300 as pkg
    pkg.lib()
    return pkg


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def check_laplace(pkg, g, mu, p, precision, layers=("slp", "dlp"), **kw):
    ref = oracle.tsqbx_laplace(g, p, mu, slp="slp" in layers, dlp="dlp" in layers)
    with pkg.Plan(g, "laplace", layers, p=p, precision=precision, **kw) as plan:
        out = plan.eval(mu)
    for layer in layers:
        e = relerr(out[layer], ref[layer])
        assert e <= TOL[precision], (layer, precision, p, e)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("p", list(range(0, 21)))
def test_laplace_every_order(pkg, precision, p):
    rng = np.random.default_rng(100 + p)
    g = cloud_geometry(rng, n_ctr=12, n_src=150, q_max=0.6, tgt_per_ctr=3, list_frac=0.7)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, p, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("lanes", [1, 2, 3, 5, 8, 16, 32])
def test_laplace_forced_lane_counts(pkg, precision, lanes):
    """Every lanes-per-target value, groups of 1..40 targets (ragged items)."""
    rng = np.random.default_rng(7)
    g = cloud_geometry(rng, n_ctr=6, n_src=300, q_max=0.5, tgt_per_ctr=40, list_frac=0.9)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, 9, precision, lanes_per_target=lanes)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("max_iters", [1, 2, 7, 40])
def test_laplace_sliced_lists(pkg, precision, max_iters):
    """Long lists cut into source slices (partials combined in slice order)."""
    rng = np.random.default_rng(31)
    g = cloud_geometry(rng, n_ctr=7, n_src=400, q_max=0.5, tgt_per_ctr=13, list_frac=0.8)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, 6, precision, max_item_iters=max_iters)
    check_laplace(pkg, g, mu, 6, precision, max_item_iters=max_iters, lanes_per_target=5)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("p,max_iters", [(0, 0), (4, 0), (9, 0), (9, 2), (13, 5)])
def test_laplace_single_target_groups(pkg, precision, p, max_iters):
    """One target per group: the direct-load path (no shared-memory staging)."""
    rng = np.random.default_rng(61 + p)
    g = cloud_geometry(rng, n_ctr=40, n_src=500, q_max=0.6, tgt_per_ctr=1, list_frac=0.5)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, p, precision, max_item_iters=max_iters)


def test_helmholtz_sliced_lists(pkg):
    rng = np.random.default_rng(37)
    g = cloud_geometry(rng, n_ctr=5, n_src=300, q_max=0.5, tgt_per_ctr=7, list_frac=0.9)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_helmholtz(g, 8, 4.0, mu)["slp"]
    for mi in (1, 5, 33):
        with pkg.Plan(g, "helmholtz", ("slp",), p=8, k=4.0, max_item_iters=mi) as plan:
            out = plan.eval(mu)["slp"]
        assert relerr(out, ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
def test_laplace_sphere_workload(pkg, precision):
    g, mu = configs.sphere()
    out = check_laplace(pkg, g, mu, 5, precision, layers=("slp",))
    assert np.all(np.isfinite(out["slp"]))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
def test_laplace_small_torus_octree_lists(pkg, precision):
    g, mu, _ = configs.torus(48, 18)
    check_laplace(pkg, g, mu, 9, precision)


def test_laplace_full_torus_sampled_targets(pkg):
    """The benchmark configuration (torus 256 x 96, octree lists, p = 9), in the
    launch configuration the benchmark times; 600 sampled targets checked
    against the oracle one by one, both precisions."""
    g, mu, _ = configs.torus()
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(g.n_tgt, 600, replace=False))
    ref = oracle.tsqbx_laplace(g, 9, mu, subset=idx, slp=True, dlp=True)
    for precision in ("fp64", "mixed", "df64"):
        with pkg.Plan(g, "laplace", ("slp", "dlp"), p=9, precision=precision) as plan:
            out = plan.eval(mu)
            info = plan.info()
        assert info["n_pairs"] == g.n_pairs() == oracle.count_pairs(g)
        for layer in ("slp", "dlp"):
            e = relerr(out[layer][idx], ref[layer])
            assert e <= TOL[precision], (precision, layer, e)


def test_edge_cases(pkg):
    rng = np.random.default_rng(11)
    # duplicated ranges are summed twice; one center with an empty list
    g = cloud_geometry(rng, n_ctr=4, n_src=60, dup=True, tgt_per_ctr=5, rho_zero=True)
    g.group_range_start = g.group_range_start.copy()
    g.range_begin, g.range_end = g.range_begin.copy(), g.range_end.copy()
    # empty list for group 0: drop its ranges
    a, b = g.group_range_start[0], g.group_range_start[1]
    keep = np.ones(len(g.range_begin), bool)
    keep[a:b] = False
    g.range_begin, g.range_end = g.range_begin[keep], g.range_end[keep]
    g.group_range_start = np.concatenate([[0, 0], g.group_range_start[2:] - (b - a)])
    mu = rng.standard_normal(g.n_src)
    out = check_laplace(pkg, g, mu, 7, "fp64")
    assert np.all(out["slp"][g.ctr_group[g.tgt_center] == 0] == 0.0)
    check_laplace(pkg, g, mu, 7, "mixed")
    check_laplace(pkg, g, mu, 7, "df64")


def test_no_targets_and_no_sources(pkg):
    rng = np.random.default_rng(5)
    g = cloud_geometry(rng, n_ctr=2, n_src=10)
    g.tgt_xyz = np.zeros((3, 0))
    g.tgt_center = np.zeros(0, np.int32)
    with pkg.Plan(g, "laplace", ("slp",), p=3) as plan:
        out = plan.eval(np.ones(g.n_src))
    assert out["slp"].shape == (0,)


def test_divergent_pairs(pkg):
    rng = np.random.default_rng(9)
    g = cloud_geometry(rng, n_ctr=2, n_src=20)
    g.tgt_xyz = g.tgt_xyz.copy()
    c = g.tgt_center[0]
    g.tgt_xyz[:, 0] = g.ctr_xyz[:, c] + 10.0        # far outside every |s-c|
    with pytest.raises(pkg.TsqbxError) as ei:
        pkg.Plan(g, "laplace", ("slp",), p=4)
    assert ei.value.code == -2
    nd, nz = oracle.count_divergent(g)
    with pkg.Plan(g, "laplace", ("slp",), p=4, allow_divergent=True) as plan:
        assert plan.info()["n_divergent"] == nd > 0
        out = plan.eval(np.ones(g.n_src))
    ref = oracle.tsqbx_laplace(g, 4, np.ones(g.n_src))["slp"]
    assert relerr(out["slp"], ref) <= 1e-12
    # a source on a center is always rejected
    h = cloud_geometry(rng, n_ctr=2, n_src=20)
    h.src_xyz = h.src_xyz.copy()
    h.src_xyz[:, h.range_begin[0]] = h.ctr_xyz[:, 0]
    with pytest.raises(pkg.TsqbxError) as ei:
        pkg.Plan(h, "laplace", ("slp",), p=4, allow_divergent=True)
    assert ei.value.code == -2


@pytest.mark.parametrize("p,k", [(0, 1.0), (4, 5.0), (12, 10.0), (12, 1.0), (20, 3.0)])
def test_helmholtz_slp(pkg, p, k):
    rng = np.random.default_rng(p + 17)
    g = cloud_geometry(rng, n_ctr=10, n_src=120, q_max=0.6, tgt_per_ctr=3, rho_zero=True)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_helmholtz(g, p, k, mu)["slp"]
    with pkg.Plan(g, "helmholtz", ("slp",), p=p, k=k) as plan:
        out = plan.eval(mu)["slp"]
    assert relerr(out, ref) <= 1e-12


@pytest.mark.parametrize("p,k", [(6, 0.01), (16, 0.01), (6, 30.0), (16, 30.0), (20, 60.0)])
def test_helmholtz_extreme_wavenumbers_all_layers(pkg, p, k):
    """The Clenshaw sums over the Hankel factors where they grow fastest (kR
    ~ 1e-2: g_n ~ (2n-1)!!/(kR)^(n+1)) and where they oscillate (kR up to
    ~100, beyond the order), for every layer combination."""
    rng = np.random.default_rng(int(10 * k) + p)
    g = cloud_geometry(rng, n_ctr=10, n_src=120, q_max=0.6, tgt_per_ctr=3, rho_zero=True)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_helmholtz(g, p, k, mu, slp=True, dlp=True, sp=True)
    for layers in (("slp",), ("dlp",), ("slp", "dlp"), ("slp", "sp"), ("slp", "dlp", "sp")):
        with pkg.Plan(g, "helmholtz", layers, p=p, k=k) as plan:
            out = plan.eval(mu)
        for layer in layers:
            assert relerr(out[layer], ref[layer]) <= 1e-12, (layers, layer)


def test_helmholtz_small_torus(pkg):
    g, mu, _ = configs.torus_helmholtz(40, 16, k=10.0)
    ref = oracle.tsqbx_helmholtz(g, 12, 10.0, mu)["slp"]
    with pkg.Plan(g, "helmholtz", ("slp",), p=12, k=10.0) as plan:
        out = plan.eval(mu)["slp"]
    assert relerr(out, ref) <= 1e-12


def test_helmholtz_full_size_torus_sampled_targets(pkg):
    """The Helmholtz workload at full size: torus 444 x 166 quads (884,448
    sources, 1,768,896 targets, octree lists), k = 10, p = 12, the single,
    double and S' layers in one plan, as the benchmark launches it; 900
    seeded random targets compared element-wise with the oracle (Appendix A,
    the Helmholtz addition theorem) at the FP64 bar."""
    g, mu, _ = configs.torus_helmholtz()
    assert g.n_src == 884448 and g.n_tgt == 1768896
    rng = np.random.default_rng(31)
    idx = np.sort(rng.choice(g.n_tgt, 900, replace=False))
    layers = ("slp", "dlp", "sp")
    ref = oracle.tsqbx_helmholtz(g, 12, 10.0, mu, subset=idx, slp=True, dlp=True, sp=True)
    with pkg.Plan(g, "helmholtz", layers, p=12, k=10.0) as plan:
        out = plan.eval(mu)
    for layer in layers:
        e = relerr(out[layer][idx], ref[layer])
        assert e <= 1e-12, (layer, e)


def test_paths_agree_and_are_deterministic(pkg):
    """Host pointers, device tensors, eval_async and submit/poll give
    bit-identical results; repeated evaluations are bit-identical."""
    import torch
    rng = np.random.default_rng(21)
    g = cloud_geometry(rng, n_ctr=20, n_src=200, tgt_per_ctr=4)
    mu = rng.standard_normal(g.n_src)
    for precision in ("fp64", "mixed", "df64"):
        with pkg.Plan(g, "laplace", ("slp", "dlp"), p=8, precision=precision) as plan:
            a = plan.eval(mu)
            b = plan.eval(mu)
            dmu = torch.from_numpy(mu).cuda()
            c = plan.eval(dmu)
            outs = {k: torch.empty(g.n_tgt, dtype=torch.float64, device="cuda") for k in ("slp", "dlp")}
            s = torch.cuda.Stream()
            plan.eval_async(dmu, outs, stream=s)
            s.synchronize()
            t, d = plan.submit(mu)
            assert pkg.poll(t, timeout_us=-1)
            for layer in ("slp", "dlp"):
                assert np.array_equal(a[layer], b[layer])
                assert np.array_equal(a[layer], c[layer].cpu().numpy())
                assert np.array_equal(a[layer], outs[layer].cpu().numpy())
                assert np.array_equal(a[layer], d[layer])


def test_submit_slots_and_busy(pkg):
    rng = np.random.default_rng(23)
    g = cloud_geometry(rng, n_ctr=8, n_src=100, tgt_per_ctr=2)
    mus = [rng.standard_normal(g.n_src) for _ in range(3)]
    with pkg.Plan(g, "laplace", ("slp",), p=5, n_slots=2) as plan:
        t1, o1 = plan.submit(mus[0])
        t2, o2 = plan.submit(mus[1])
        with pytest.raises(pkg.TsqbxError) as ei:
            plan.submit(mus[2])
        assert ei.value.code == -6
        assert pkg.poll(t1, -1) and pkg.poll(t2, -1)
        with pytest.raises(pkg.TsqbxError) as ei:
            pkg.poll(t1, 0)
        assert ei.value.code == -7
        for mu, o in zip(mus[:2], (o1, o2)):
            ref = oracle.tsqbx_laplace(g, 5, mu)["slp"]
            assert relerr(o["slp"], ref) <= 1e-12


def ragged_range_geometry(rng, n_src=600, n_ctr=9, tgt_per_ctr=(1, 5, 17)):
    """Groups whose ranges abut (so they merge into one run), include empty
    ranges, run backwards through the source order, repeat a source range,
    or are empty altogether; targets as in cloud_geometry (convergent).
    Sources lie in a shell with outward normals, so that with a positive
    density the layers are as well conditioned as on a surface."""
    from tsqbx_inputs.geometry import Geometry
    src = rng.uniform(-2, 2, (4 * n_src, 3))
    src = src[np.linalg.norm(src, axis=1) >= 0.9][:n_src]     # >= 0.2 from every center
    w = rng.uniform(0.5, 1.5, n_src)
    nrm = src / np.linalg.norm(src, axis=1, keepdims=True)     # outward, like a closed surface's
    ctr = rng.uniform(-0.4, 0.4, (n_ctr, 3))
    rb, re, grs = [], [], [0]
    for c in range(n_ctr):
        kind = c % 5
        if kind == 0:          # one long run cut into abutting pieces, with empty ranges between
            a = int(rng.integers(0, 100))
            cuts = np.sort(rng.choice(np.arange(a + 1, a + 450), size=12, replace=False))
            edges = [a] + list(cuts) + [a + 450]
            for lo, hi in zip(edges[:-1], edges[1:]):
                rb.append(lo); re.append(hi)
                rb.append(hi); re.append(hi)                     # empty
        elif kind == 1:        # runs in decreasing source order
            for lo in range(540, 0, -60):
                rb.append(lo); re.append(lo + int(rng.integers(1, 40)))
        elif kind == 2:        # the same range twice, and a single source
            rb += [10, 10, 333]; re += [210, 210, 334]
        elif kind == 3:        # nothing but empty ranges
            rb += [5, 70]; re += [5, 70]
        else:                  # many one-source runs
            sel = np.sort(rng.choice(n_src, size=120, replace=False))
            rb += list(sel); re += list(sel + 1)
        grs.append(len(rb))
    rb, re, grs = np.array(rb, np.int32), np.array(re, np.int32), np.array(grs, np.int64)
    tgt, tc, tn = [], [], []
    for c in range(n_ctr):
        members = [np.arange(rb[i], re[i]) for i in range(grs[c], grs[c + 1])]
        members = np.concatenate(members) if members else np.zeros(0, int)
        Rmin = np.linalg.norm(src[members] - ctr[c], axis=1).min() if len(members) else 1.0
        for j in range(tgt_per_ctr[c % len(tgt_per_ctr)]):
            d = rng.standard_normal(3)
            tgt.append(ctr[c] + rng.uniform(0.05, 0.6) * Rmin * d / np.linalg.norm(d))
            tc.append(c)
            tn.append(d / np.linalg.norm(d))
    tgt = np.array(tgt)
    return Geometry(np.ascontiguousarray(src.T), w, np.ascontiguousarray(nrm.T), np.ascontiguousarray(ctr.T),
                    np.full(n_ctr, 0.1), np.ascontiguousarray(tgt.T), np.array(tc, np.int32),
                    np.ascontiguousarray(np.array(tn).T), np.arange(n_ctr, dtype=np.int32), grs, rb, re)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("max_iters,lanes", [(0, 0), (1, 0), (2, 3), (3, 32), (0, 1)])
def test_laplace_ragged_range_lists(pkg, precision, max_iters, lanes):
    """Source lists read as merged runs: abutting, empty, backwards, repeated
    and single-source ranges, slices that start inside a run, every path."""
    rng = np.random.default_rng(2024 + max_iters)
    g = ragged_range_geometry(rng)
    mu = 1.0 + 0.5 * rng.uniform(-1, 1, g.n_src)
    out = check_laplace(pkg, g, mu, 7, precision, max_item_iters=max_iters, lanes_per_target=lanes)
    empty = g.tgt_center % 5 == 3
    assert np.all(out["slp"][empty] == 0.0) and np.all(out["dlp"][empty] == 0.0)


def test_helmholtz_ragged_range_lists(pkg):
    rng = np.random.default_rng(77)
    g = ragged_range_geometry(rng)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_helmholtz(g, 8, 4.0, mu, slp=True, dlp=True)
    for max_iters in (0, 2):
        with pkg.Plan(g, "helmholtz", ("slp", "dlp"), p=8, k=4.0, max_item_iters=max_iters) as plan:
            out = plan.eval(mu)
        for layer in ("slp", "dlp"):
            assert relerr(out[layer], ref[layer]) <= 1e-12, (layer, max_iters)
