"""Full-size parity for the two systems workloads, in the launch configuration
the benchmark times, on outputs the oracle computes one by one.

* The batched workload: 64 seeded ellipsoids (1k-200k sources each, 2.09M in
  all), Laplace single layer, p in {5, 7, 9}, mixed precision, every plan in
  one persistent launch replayed from a CUDA graph.  Sampled targets of every
  surface against the FP64 oracle (Sec. 3, the target-specific expansion) at
  the mixed bar, and two replays bit-identical.
* The serving workload: the 16 resident geometries (5k-300k sources), every
  request kind the benchmark draws (Laplace FP64 served by the double-float
  kernels, Laplace mixed, Helmholtz k = 1, 5, 10) at p = 5, 9, 12, submitted
  together so that they run concurrently and the Helmholtz ones merge;
  sampled targets of every result against the oracle at the bar of its
  precision."""
import numpy as np
import pytest

import oracle

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


def test_batched_workload_full_size(env):
    torch, pkg = env
    from tsqbx_inputs import configs
    surfaces = configs.ellipsoid_batch()
    assert len(surfaces) == 64
    assert sum(g.n_src for g, _ in surfaces) > 2_000_000
    plans = [pkg.Plan(g, "laplace", ("slp",), p=g.meta["p"], precision="mixed") for g, _ in surfaces]
    try:
        dens = [torch.from_numpy(mu).cuda() for _, mu in surfaces]
        runs = []
        with pkg.Batch(plans, use_graph=True) as batch:
            for _ in range(2):
                outs = [{"slp": torch.full((g.n_tgt,), np.nan, dtype=torch.float64, device="cuda")}
                        for g, _ in surfaces]
                batch.eval_async(dens, outs, stream=torch.cuda.current_stream())
                torch.cuda.synchronize()
                runs.append([o["slp"].cpu().numpy() for o in outs])
        for a, b in zip(*runs):
            assert np.array_equal(a, b)
        rng = np.random.default_rng(2024)
        for i, (g, mu) in enumerate(surfaces):
            idx = np.sort(rng.choice(g.n_tgt, min(40, g.n_tgt), replace=False))
            ref = oracle.tsqbx_laplace(g, g.meta["p"], mu, subset=idx)["slp"]
            e = relerr(runs[0][i][idx], ref)
            assert e <= 1e-6, (i, e)
    finally:
        for p_ in plans:
            p_.close()


def test_serving_workload_full_size(env):
    torch, pkg = env
    from tsqbx_inputs import configs
    geoms = configs.serving_geometries()
    assert len(geoms) == 16
    kinds = [("laplace", "fp64", 0.0, 1e-12), ("laplace", "mixed", 0.0, 1e-6),
             ("helmholtz", "fp64", 1.0, 1e-12), ("helmholtz", "fp64", 5.0, 1e-12),
             ("helmholtz", "fp64", 10.0, 1e-12)]
    rng = np.random.default_rng(2025)
    reqs = []
    with pkg.Server(hbm_budget=64 << 30, max_inflight=64, laplace_fp64_path="df64") as srv:
        gids = [srv.add_geometry(g, with_normals=False) for g in geoms]
        for n, (gi, g) in enumerate(zip(gids, geoms)):
            for m, (kernel, prec, k, tol) in enumerate(kinds):
                p = (5, 9, 12)[(n + m) % 3]
                mu = rng.standard_normal(g.n_src)
                if kernel == "helmholtz":
                    mu = mu + 1j * rng.standard_normal(g.n_src)
                rid, outs = srv.submit(gi, mu, kernel, ("slp",), p, k, prec)
                reqs.append((rid, outs, n, kernel, p, k, mu, tol))
            # a second Helmholtz request of the same plan, order and wavenumber,
            # which may start merged with the first
            mu2 = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
            rid, outs = srv.submit(gi, mu2, "helmholtz", ("slp",), 12, 10.0, "fp64")
            reqs.append((rid, outs, n, "helmholtz", 12, 10.0, mu2, 1e-12))
        for rid, *_ in reqs:
            assert srv.poll(rid, -1)
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["rejected"] == 0
    for rid, outs, n, kernel, p, k, mu, tol in reqs:
        g = geoms[n]
        idx = np.sort(rng.choice(g.n_tgt, min(30, g.n_tgt), replace=False))
        if kernel == "laplace":
            ref = oracle.tsqbx_laplace(g, p, mu, subset=idx)["slp"]
        else:
            ref = oracle.tsqbx_helmholtz(g, p, k, mu, subset=idx)["slp"]
        e = relerr(outs["slp"][idx], ref)
        assert e <= tol, (n, kernel, p, k, e)
