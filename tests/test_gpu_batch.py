"""Batched persistent launch (tsqbx_batch_*): many plans of uneven size and
order in one launch give exactly the per-plan results."""
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


def _geoms(seed):
    rng = np.random.default_rng(seed)
    spec = [(3, 40, 2, 3), (9, 300, 5, 5), (25, 900, 8, 9), (1, 50, 1, 0), (14, 500, 3, 7)]
    out = []
    for n_ctr, n_src, tpc, p in spec:
        g = cloud_geometry(rng, n_ctr=n_ctr, n_src=n_src, q_max=0.5, tgt_per_ctr=tpc, list_frac=0.7)
        out.append((g, rng.standard_normal(g.n_src), p))
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_individual_plans(env, precision, tol, use_graph):
    torch, pkg = env
    items = _geoms(51)
    plans = [pkg.Plan(g, "laplace", ("slp", "dlp"), p=p, precision=precision,
                      max_item_iters=3 if i == 2 else 0) for i, (g, mu, p) in enumerate(items)]
    try:
        with pkg.Batch(plans, use_graph=use_graph) as batch:
            info = batch.info()
            assert info["n_plans"] == len(plans) and info["graph"] == int(use_graph)
            assert info["n_sliced"] > 0
            for rep in range(2):                      # replay with new densities
                dens, outs = [], []
                for g, mu, p in items:
                    m = mu * (1.0 + rep)
                    dens.append(torch.from_numpy(m).cuda())
                    outs.append({l: torch.full((g.n_tgt,), np.nan, dtype=torch.float64, device="cuda")
                                 for l in ("slp", "dlp")})
                batch.eval_async(dens, outs, stream=torch.cuda.current_stream())
                assert batch.kernel_ms() > 0
                for (g, mu, p), plan, o, d in zip(items, plans, outs, dens):
                    single = plan.eval(d)
                    ref = oracle.tsqbx_laplace(g, p, mu * (1.0 + rep), slp=True, dlp=True)
                    for l in ("slp", "dlp"):
                        got = o[l].cpu().numpy()
                        assert np.array_equal(got, single[l].cpu().numpy()), (l, p)
                        err = np.max(np.abs(got - ref[l])) / np.max(np.abs(ref[l]))
                        assert err <= tol
    finally:
        for p_ in plans:
            p_.close()


def test_batch_rejects_mixed_kinds(env):
    torch, pkg = env
    (g1, _, _), (g2, _, _) = _geoms(53)[:2]
    a = pkg.Plan(g1, "laplace", ("slp",), p=3, precision="fp64")
    b = pkg.Plan(g2, "laplace", ("slp",), p=3, precision="mixed")
    h = pkg.Plan(g2, "helmholtz", ("slp",), p=3, k=2.0)
    try:
        with pytest.raises(pkg.TsqbxError) as ei:
            pkg.Batch([a, b])
        assert ei.value.code == -1
        with pytest.raises(pkg.TsqbxError) as ei:
            pkg.Batch([h])
        assert ei.value.code == -9
    finally:
        for p_ in (a, b, h):
            p_.close()


def test_single_layer_mixed_batch_shared_warp_items(env):
    """Single-target items of one plan run up to four per warp (8 or 16 lanes
    each) in single-layer mixed batches: results within 1e-6 of the oracle
    and of each plan alone (the lanes reduce in another order), and
    bit-identical from one replay to the next."""
    torch, pkg = env
    from tsqbx_inputs import configs
    items = configs.ellipsoid_batch(n_surfaces=6, max_src=20000)
    plans = [pkg.Plan(g, "laplace", ("slp",), p=g.meta["p"], precision="mixed") for g, mu in items]
    try:
        with pkg.Batch(plans) as batch:
            runs = []
            for rep in range(2):
                dens = [torch.from_numpy(mu).cuda() for g, mu in items]
                outs = [{"slp": torch.full((g.n_tgt,), np.nan, dtype=torch.float64, device="cuda")}
                        for g, mu in items]
                batch.eval_async(dens, outs, stream=torch.cuda.current_stream())
                torch.cuda.synchronize()
                runs.append([o["slp"].cpu().numpy() for o in outs])
            for a, b in zip(*runs):
                assert np.array_equal(a, b)
            for (g, mu), plan, got in zip(items, plans, runs[0]):
                single = plan.eval(mu)["slp"]
                assert np.max(np.abs(got - single)) / np.max(np.abs(single)) <= 1e-6
                idx = np.sort(np.random.default_rng(1).choice(g.n_tgt, min(300, g.n_tgt), replace=False))
                ref = oracle.tsqbx_laplace(g, g.meta["p"], mu, subset=idx)["slp"]
                assert np.max(np.abs(got[idx] - ref)) / np.max(np.abs(ref)) <= 1e-6
    finally:
        for p_ in plans:
            p_.close()


def test_window_items_with_a_source_on_a_neighbours_center(env):
    """Four consecutive single-target items whose lists are overlapping windows
    of consecutive sources share one staged union in a single-layer mixed
    batch.  A source inside the union sits exactly on the first center but
    outside that center's own window: it must contribute nothing there (no
    inf/NaN), and every result must match the oracle within 1e-6."""
    torch, pkg = env
    from tsqbx_inputs.geometry import Geometry
    rng = np.random.default_rng(71)
    n_src, n_ctr, width, step = 130, 8, 50, 10
    t = np.linspace(0.0, 2.0, n_src)
    src = np.stack([t, 0.3 * np.sin(3 * t), 0.2 * np.cos(2 * t)])
    ctr = np.stack([np.linspace(0.2, 1.2, n_ctr), np.full(n_ctr, 0.6), np.full(n_ctr, 0.5)])
    src[:, 55] = ctr[:, 0]                                   # in centers 1-4's windows, not in center 0's
    begin = np.arange(n_ctr, dtype=np.int32) * step
    end = begin + width
    d = rng.standard_normal((3, n_ctr))
    d /= np.linalg.norm(d, axis=0)
    rmin = np.array([np.linalg.norm(src[:, b:e] - ctr[:, [c]], axis=0).min()
                     for c, (b, e) in enumerate(zip(begin, end))])
    tgt = ctr + 0.3 * rmin * d
    g = Geometry(np.ascontiguousarray(src), rng.uniform(0.5, 1.5, n_src), None, np.ascontiguousarray(ctr),
                 np.full(n_ctr, 0.1), np.ascontiguousarray(tgt), np.arange(n_ctr, dtype=np.int32), None,
                 np.arange(n_ctr, dtype=np.int32), np.arange(n_ctr + 1, dtype=np.int64), begin, end)
    mu = rng.standard_normal(n_src)
    plan = pkg.Plan(g, "laplace", ("slp",), p=7, precision="mixed")
    try:
        with pkg.Batch([plan]) as batch:
            dmu = torch.from_numpy(mu).cuda()
            out = {"slp": torch.full((n_ctr,), np.nan, dtype=torch.float64, device="cuda")}
            batch.eval_async([dmu], [out], stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
            got = out["slp"].cpu().numpy()
    finally:
        plan.close()
    ref = oracle.tsqbx_laplace(g, 7, mu, slp=True)["slp"]
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-6


def test_batch_of_plans_with_tuned_order_forms(env):
    """Plans whose own evaluations use the runtime-order kernel (p_unroll)
    still batch: the persistent launch runs the per-order item bodies for
    every plan, within the FP64 bar of the oracle and of each plan alone.
    Double-float plans do not batch (the persistent kernel has no
    double-float body)."""
    torch, pkg = env
    items = _geoms(57)
    plans = [pkg.Plan(g, "laplace", ("slp", "dlp"), p=p, precision="fp64", p_unroll=(1, 2, 4, 0, 2)[i])
             for i, (g, mu, p) in enumerate(items)]
    try:
        with pkg.Batch(plans) as batch:
            dens = [torch.from_numpy(mu).cuda() for g, mu, p in items]
            outs = [{l: torch.full((g.n_tgt,), np.nan, dtype=torch.float64, device="cuda") for l in ("slp", "dlp")}
                    for g, mu, p in items]
            batch.eval_async(dens, outs, stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
        for (g, mu, p), plan, o in zip(items, plans, outs):
            alone = plan.eval(mu)
            ref = oracle.tsqbx_laplace(g, p, mu, slp=True, dlp=True)
            for l in ("slp", "dlp"):
                got = o[l].cpu().numpy()
                assert np.max(np.abs(got - ref[l])) / np.max(np.abs(ref[l])) <= 1e-12
                assert np.max(np.abs(got - alone[l])) / np.max(np.abs(alone[l])) <= 1e-13
    finally:
        for p_ in plans:
            p_.close()
    g, mu, p = items[0]
    with pkg.Plan(g, "laplace", ("slp",), p=p, precision="df64") as dfp:
        with pytest.raises(pkg.TsqbxError) as e:
            pkg.Batch([dfp])
        assert e.value.code == -9
