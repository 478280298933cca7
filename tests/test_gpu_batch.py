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
