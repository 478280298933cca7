"""GPU parity for the conventional QBX path (coefficient formation per center,
then evaluation per target; Sec. 2.1 eqs. local-coeffs and local-expansion),
through the C ABI, against the FP64 oracle's conventional path (path B) and
its target-specific path (path A): both define the same truncated expansion.
Tolerance 1e-12 relative in the max norm (FP64)."""
import numpy as np
import pytest

import oracle
from helpers import cloud_geometry

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


def run(pkg, g, mu, p, layers, conventional, **kw):
    with pkg.Plan(g, "laplace", layers, p=p, conventional=conventional, **kw) as plan:
        out = plan.eval(mu)
        info = plan.info()
    return out, info


@pytest.mark.parametrize("p", list(range(0, 21)))
def test_all_conventional_every_order(pkg, p):
    rng = np.random.default_rng(500 + p)
    g = cloud_geometry(rng, n_ctr=6, n_src=90, q_max=0.6, tgt_per_ctr=5, list_frac=0.8)
    mu = rng.standard_normal(g.n_src)
    out, info = run(pkg, g, mu, p, ("slp", "dlp", "sp"), "all")
    assert info["n_conv_centers"] == 6 and info["n_conv_targets"] == g.n_tgt
    ref_b = oracle.qbx_laplace(g, p, mu, slp=True, dlp=True, sp=True)
    ref_a = oracle.tsqbx_laplace(g, p, mu, slp=True, dlp=True, sp=True)
    for layer in ("slp", "dlp", "sp"):
        assert relerr(out[layer], ref_b[layer]) <= TOL, (layer, p)
        assert relerr(out[layer], ref_a[layer]) <= TOL, (layer, p)


@pytest.mark.parametrize("layers", [("slp",), ("dlp",), ("sp",), ("slp", "dlp"), ("dlp", "sp")])
def test_layer_subsets(pkg, layers):
    rng = np.random.default_rng(71)
    g = cloud_geometry(rng, n_ctr=5, n_src=120, q_max=0.5, tgt_per_ctr=9, list_frac=0.9)
    mu = rng.standard_normal(g.n_src)
    out, _ = run(pkg, g, mu, 8, layers, "all")
    ref = oracle.tsqbx_laplace(g, 8, mu, slp=True, dlp="dlp" in layers, sp="sp" in layers)
    assert set(out) == set(layers)
    for layer in layers:
        assert relerr(out[layer], ref[layer]) <= TOL, layer


def test_long_lists_many_slices_and_targets(pkg):
    """Lists longer than one coefficient slice (1024 sources) and centers with
    more than 32 targets (several evaluation items per center)."""
    rng = np.random.default_rng(73)
    g = cloud_geometry(rng, n_ctr=3, n_src=2600, q_max=0.5, tgt_per_ctr=70, list_frac=0.95)
    mu = rng.standard_normal(g.n_src)
    out, info = run(pkg, g, mu, 7, ("slp", "dlp"), "all")
    assert info["n_conv_items"] >= 9
    ref = oracle.tsqbx_laplace(g, 7, mu, slp=True, dlp=True)
    for layer in ("slp", "dlp"):
        assert relerr(out[layer], ref[layer]) <= TOL, layer


def test_target_on_center_and_empty_list(pkg):
    rng = np.random.default_rng(79)
    g = cloud_geometry(rng, n_ctr=4, n_src=60, tgt_per_ctr=6, rho_zero=True)
    a, b = g.group_range_start[0], g.group_range_start[1]
    keep = np.ones(len(g.range_begin), bool)
    keep[a:b] = False
    g.range_begin, g.range_end = g.range_begin[keep], g.range_end[keep]
    g.group_range_start = np.concatenate([[0, 0], g.group_range_start[2:] - (b - a)])
    mu = rng.standard_normal(g.n_src)
    out, _ = run(pkg, g, mu, 6, ("slp", "dlp", "sp"), "all")
    ref = oracle.tsqbx_laplace(g, 6, mu, slp=True, dlp=True, sp=True)
    for layer in ("slp", "dlp", "sp"):
        assert relerr(out[layer], ref[layer]) <= TOL, layer
    assert np.all(out["slp"][g.ctr_group[g.tgt_center] == 0] == 0.0)


def test_auto_mixes_paths(pkg):
    """The cost model sends centers with many targets to the conventional path
    and the rest to the target-specific one; results agree either way."""
    rng = np.random.default_rng(83)
    g = cloud_geometry(rng, n_ctr=8, n_src=400, q_max=0.5, tgt_per_ctr=1, list_frac=0.9)
    # give centers 0 and 1 forty extra targets each, no farther from the
    # center than its first target (so inside the convergence ball)
    extra_t, extra_c, extra_n = [], [], []
    for c in (0, 1):
        ctr = g.ctr_xyz[:, c]
        rho = np.linalg.norm(g.tgt_xyz[:, np.flatnonzero(g.tgt_center == c)[0]] - ctr)
        for j in range(40):
            v = rng.standard_normal(3)
            v /= np.linalg.norm(v)
            extra_t.append(ctr + rng.uniform(0.2, 1.0) * rho * v)
            extra_c.append(c)
            extra_n.append(v)
    g.tgt_xyz = np.ascontiguousarray(np.concatenate([g.tgt_xyz, np.array(extra_t).T], axis=1))
    g.tgt_center = np.concatenate([g.tgt_center, np.array(extra_c, np.int32)])
    g.tgt_normal = np.ascontiguousarray(np.concatenate([g.tgt_normal, np.array(extra_n).T], axis=1))
    mu = rng.standard_normal(g.n_src)
    out, info = run(pkg, g, mu, 9, ("slp", "dlp"), "auto")
    assert info["n_conv_centers"] == 2 and info["n_conv_targets"] == 82
    ref = oracle.tsqbx_laplace(g, 9, mu, slp=True, dlp=True)
    for layer in ("slp", "dlp"):
        assert relerr(out[layer], ref[layer]) <= TOL, layer
    ts, _ = run(pkg, g, mu, 9, ("slp", "dlp"), "off")
    for layer in ("slp", "dlp"):
        assert relerr(out[layer], ts[layer]) <= TOL, layer


def test_deterministic_and_per_call_order(pkg):
    import torch
    rng = np.random.default_rng(89)
    g = cloud_geometry(rng, n_ctr=5, n_src=300, tgt_per_ctr=12)
    mu = rng.standard_normal(g.n_src)
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=10, conventional="all") as plan:
        a = plan.eval(mu)
        b = plan.eval(torch.from_numpy(mu).cuda())
        c = plan.eval(mu, p=4)
        with pytest.raises(pkg.TsqbxError) as ei:
            plan.eval(mu, p=11)
        assert ei.value.code == -9
    for layer in ("slp", "dlp"):
        assert np.array_equal(a[layer], b[layer].cpu().numpy())
    ref4 = oracle.tsqbx_laplace(g, 4, mu, slp=True, dlp=True)
    for layer in ("slp", "dlp"):
        assert relerr(c[layer], ref4[layer]) <= TOL


def test_unsupported_combinations(pkg):
    rng = np.random.default_rng(97)
    g = cloud_geometry(rng, n_ctr=2, n_src=30, tgt_per_ctr=3)
    for kw in (dict(precision="mixed"), dict(precision="df64")):
        with pytest.raises(pkg.TsqbxError) as ei:
            kernel = kw.pop("kernel", "laplace")
            pkg.Plan(g, kernel, ("slp",), p=4, conventional="all", **kw)
        assert ei.value.code == -9


# ------------------------------------------------------------------ Helmholtz

@pytest.mark.parametrize("p,k", [(0, 1.0), (1, 2.0), (4, 5.0), (8, 0.5), (10, 3.0), (12, 10.0)])
def test_helmholtz_all_conventional(pkg, p, k):
    rng = np.random.default_rng(600 + p)
    g = cloud_geometry(rng, n_ctr=6, n_src=90, q_max=0.6, tgt_per_ctr=5, list_frac=0.8, rho_zero=True)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    with pkg.Plan(g, "helmholtz", ("slp", "dlp", "sp"), p=p, k=k, conventional="all") as plan:
        out = plan.eval(mu)
        assert plan.info()["n_conv_centers"] == 6
    ref_a = oracle.tsqbx_helmholtz(g, p, k, mu, slp=True, dlp=True, sp=True)
    ref_b = oracle.qbx_helmholtz(g, p, k, mu, slp=True, dlp=True, sp=True)
    for layer in ("slp", "dlp", "sp"):
        assert relerr(out[layer], ref_a[layer]) <= TOL, (layer, p)
        assert relerr(out[layer], ref_b[layer]) <= TOL, (layer, p)


@pytest.mark.parametrize("layers", [("slp",), ("dlp",), ("sp",), ("slp", "dlp"), ("dlp", "sp")])
def test_helmholtz_layer_subsets(pkg, layers):
    rng = np.random.default_rng(611)
    g = cloud_geometry(rng, n_ctr=5, n_src=120, q_max=0.5, tgt_per_ctr=7, list_frac=0.9)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    with pkg.Plan(g, "helmholtz", layers, p=7, k=4.0, conventional="all") as plan:
        out = plan.eval(mu)
    ref = oracle.tsqbx_helmholtz(g, 7, 4.0, mu, slp=True, dlp="dlp" in layers, sp="sp" in layers)
    for layer in layers:
        assert relerr(out[layer], ref[layer]) <= TOL, layer


def test_helmholtz_long_lists_and_targets(pkg):
    rng = np.random.default_rng(613)
    g = cloud_geometry(rng, n_ctr=3, n_src=2200, q_max=0.5, tgt_per_ctr=45, list_frac=0.95)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    with pkg.Plan(g, "helmholtz", ("slp", "dlp"), p=9, k=6.0, conventional="all") as plan:
        out = plan.eval(mu)
        assert plan.info()["n_conv_items"] >= 6
    ref = oracle.tsqbx_helmholtz(g, 9, 6.0, mu, slp=True, dlp=True)
    for layer in ("slp", "dlp"):
        assert relerr(out[layer], ref[layer]) <= TOL, layer


def test_helmholtz_order_cap(pkg):
    rng = np.random.default_rng(617)
    g = cloud_geometry(rng, n_ctr=3, n_src=60, tgt_per_ctr=20)
    with pytest.raises(pkg.TsqbxError) as ei:
        pkg.Plan(g, "helmholtz", ("slp",), p=13, k=2.0, conventional="all")
    assert ei.value.code == -9
    with pkg.Plan(g, "helmholtz", ("slp",), p=13, k=2.0, conventional="auto") as plan:
        assert plan.info()["n_conv_centers"] == 0


def test_helmholtz_auto_and_per_call(pkg):
    """Many targets per center: the cost model takes the conventional path;
    per-call order and wavenumber below the plan's."""
    rng = np.random.default_rng(619)
    g = cloud_geometry(rng, n_ctr=4, n_src=500, q_max=0.5, tgt_per_ctr=120, list_frac=0.9)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    with pkg.Plan(g, "helmholtz", ("slp",), p=10, k=3.0, conventional="auto") as plan:
        assert plan.info()["n_conv_centers"] == 4
        out = plan.eval(mu)
        out2 = plan.eval(mu, p=6, k=1.5)
    assert relerr(out["slp"], oracle.tsqbx_helmholtz(g, 10, 3.0, mu)["slp"]) <= TOL
    assert relerr(out2["slp"], oracle.tsqbx_helmholtz(g, 6, 1.5, mu)["slp"]) <= TOL


@pytest.mark.parametrize("kernel", ["laplace", "helmholtz"])
def test_auto_on_torus_with_mixed_target_counts(pkg, kernel):
    """Octree groups whose centers hold 1..64 targets: the cost model splits
    the centers of one group between the two paths; the result matches the
    target-specific path everywhere and the oracle on sampled targets."""
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus_near_targets(32, 12, "mixed:64")
    kw = {}
    if kernel == "helmholtz":
        mu = mu * np.exp(1j * 4.0 * g.src_xyz[0])
        kw = {"k": 4.0}
    layers = ("slp", "dlp", "sp")
    with pkg.Plan(g, kernel, layers, p=8, conventional="auto", **kw) as plan:
        out = plan.eval(mu)
        info = plan.info()
    assert 0 < info["n_conv_centers"] < g.n_ctr
    cnt = np.bincount(g.tgt_center, minlength=g.n_ctr)
    assert info["n_conv_targets"] > np.sum(cnt[cnt < 4])     # the conventional centers are the busy ones
    with pkg.Plan(g, kernel, layers, p=8, conventional="off", **kw) as plan:
        ts = plan.eval(mu)
    for layer in layers:
        assert relerr(out[layer], ts[layer]) <= TOL, layer
    idx = np.sort(np.random.default_rng(5).choice(g.n_tgt, 300, replace=False))
    if kernel == "laplace":
        ref = oracle.tsqbx_laplace(g, 8, mu, subset=idx, slp=True, dlp=True, sp=True)
    else:
        ref = oracle.tsqbx_helmholtz(g, 8, 4.0, mu, subset=idx, slp=True, dlp=True, sp=True)
    for layer in layers:
        assert relerr(out[layer][idx], ref[layer]) <= TOL, layer
