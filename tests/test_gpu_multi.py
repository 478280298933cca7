"""Several densities in one evaluation (tsqbx_submit_multi_layers): the
single layer (Appendix A) of the Helmholtz kernel, and the single and double
layers of the Laplace kernel in FP64 and double-float, for up to four
densities sharing every per-pair quantity.  Each result must be
bit-identical to the evaluation of its density alone on the same plan, and
within the FP64 bar (1e-12) of the oracle; sliced lists (partial sums
combined per density and layer), every staging depth, single-target and
multi-target items, both Laplace FP64 order forms, the double-float plans'
FP64 share, host and device buffers are covered.  The serving loop merges
queued requests of one plan, order and (Helmholtz) wavenumber this way."""
import ctypes

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


def _densities(rng, n_src, n):
    return [rng.standard_normal(n_src) + 1j * rng.standard_normal(n_src) for _ in range(n)]


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("p,k", [(0, 1.0), (5, 3.0), (12, 10.0), (20, 2.0)])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_multi_equals_each_density_alone(pkg, p, k, n):
    rng = np.random.default_rng(100 * p + n)
    g = cloud_geometry(rng, n_ctr=10, n_src=180, q_max=0.6, tgt_per_ctr=4, list_frac=0.7)
    dens = _densities(rng, g.n_src, n)
    with pkg.Plan(g, "helmholtz", ("slp",), p=p, k=k, max_rhs=4) as plan:
        t, outs = plan.submit_multi(dens)
        assert pkg.poll(t, -1)
        for d, o in zip(dens, outs):
            alone = plan.eval(d)["slp"]
            assert np.array_equal(o["slp"], alone)
    ref = oracle.tsqbx_helmholtz(g, p, k, dens[-1], slp=True)["slp"]
    assert _relerr(outs[-1]["slp"], ref) <= 1e-12


@pytest.mark.parametrize("depth", [32, 64, 128])
@pytest.mark.parametrize("max_iters", [0, 2])
def test_multi_sliced_lists_and_depths(pkg, depth, max_iters):
    """Sliced lists: each density's partial sums are combined on their own."""
    rng = np.random.default_rng(7 + depth + max_iters)
    g = cloud_geometry(rng, n_ctr=6, n_src=400, q_max=0.5, tgt_per_ctr=9, list_frac=0.8)
    dens = _densities(rng, g.n_src, 3)
    with pkg.Plan(g, "helmholtz", ("slp",), p=9, k=4.0, max_rhs=3, tile_depth=depth,
                  max_item_iters=max_iters) as plan:
        if max_iters:
            assert plan.info()["n_sliced"] > 0
        t, outs = plan.submit_multi(dens, p=7, k=5.0)
        assert pkg.poll(t, -1)
        for d, o in zip(dens, outs):
            assert np.array_equal(o["slp"], plan.eval(d, p=7, k=5.0)["slp"])
            ref = oracle.tsqbx_helmholtz(g, 7, 5.0, d, slp=True)["slp"]
            assert _relerr(o["slp"], ref) <= 1e-12


def test_multi_device_buffers_and_slot_reuse(pkg):
    import torch
    rng = np.random.default_rng(11)
    g = cloud_geometry(rng, n_ctr=8, n_src=200, tgt_per_ctr=5)
    dens = _densities(rng, g.n_src, 4)
    with pkg.Plan(g, "helmholtz", ("slp",), p=8, k=2.5, max_rhs=4, n_slots=2) as plan:
        ddev = [torch.from_numpy(d).cuda() for d in dens]
        t1, o1 = plan.submit_multi(ddev)                       # device in, device out
        t2, o2 = plan.submit_multi(dens[:2])                   # host, on the other slot
        assert pkg.poll(t1, -1) and pkg.poll(t2, -1)
        t3, o3 = plan.submit(dens[3])                          # a single-density call after a multi one
        assert pkg.poll(t3, -1)
        for i in range(4):
            alone = plan.eval(dens[i])["slp"]
            assert np.array_equal(o1[i]["slp"].cpu().numpy(), alone)
            if i < 2:
                assert np.array_equal(o2[i]["slp"], alone)
        assert np.array_equal(o3["slp"], plan.eval(dens[3])["slp"])


def test_multi_argument_checks(pkg):
    from paper_1811_01110_gb300 import _lib
    rng = np.random.default_rng(13)
    g = cloud_geometry(rng, n_ctr=4, n_src=60, tgt_per_ctr=2)
    dens = _densities(rng, g.n_src, 3)
    with pytest.raises(pkg.TsqbxError) as e:                     # a mixed Laplace plan cannot hold several
        pkg.Plan(g, "laplace", ("slp",), p=4, precision="mixed", max_rhs=2)
    assert e.value.code == _lib.TSQBX_E_UNSUPPORTED
    with pytest.raises(pkg.TsqbxError) as e:                     # nor a Helmholtz double layer
        pkg.Plan(g, "helmholtz", ("slp", "dlp"), p=4, k=1.0, max_rhs=2)
    assert e.value.code == _lib.TSQBX_E_UNSUPPORTED
    with pkg.Plan(g, "helmholtz", ("slp",), p=4, k=1.0, max_rhs=2) as plan:
        with pytest.raises(pkg.TsqbxError) as e:                 # more densities than max_rhs
            plan.submit_multi(dens)
        assert e.value.code == _lib.TSQBX_E_INVAL
    with pkg.Plan(g, "helmholtz", ("slp",), p=4, k=1.0) as plan:  # max_rhs 0 = 1
        with pytest.raises(pkg.TsqbxError) as e:
            plan.submit_multi(dens[:2])
        assert e.value.code == _lib.TSQBX_E_INVAL
    with pkg.Plan(g, "helmholtz", ("slp",), p=4, k=1.0, max_rhs=2, conventional="all") as plan:
        with pytest.raises(pkg.TsqbxError) as e:
            plan.submit_multi(dens[:2])
        assert e.value.code == _lib.TSQBX_E_UNSUPPORTED


def test_server_merges_queued_requests(pkg):
    """A burst of Helmholtz single-layer requests for one geometry, order and
    wavenumber: while the plan's slots are busy the rest queue, and they start
    together in multi-density evaluations.  Every result equals the request
    evaluated alone, bit for bit, and the oracle within 1e-12."""
    from tsqbx_inputs import configs
    g, _ = configs.sphere(subdiv=2)
    rng = np.random.default_rng(17)
    dens = _densities(rng, g.n_src, 16)
    with pkg.Server(hbm_budget=4 << 30, max_inflight=8) as srv:
        gid = srv.add_geometry(g)
        reqs = [srv.submit(gid, d, "helmholtz", ("slp",), 12, 10.0) for d in dens]
        for rid, _ in reqs:
            assert srv.poll(rid, -1)
        st = srv.stats()
    assert st["completed"] == len(dens) and st["failed"] == 0
    assert st["merged"] > 0
    with pkg.Plan(g, "helmholtz", ("slp",), p=12, k=10.0) as alone:
        for d, (rid, outs) in zip(dens, reqs):
            assert np.array_equal(outs["slp"], alone.eval(d)["slp"])
    ref = oracle.tsqbx_helmholtz(g, 12, 10.0, dens[5], slp=True)["slp"]
    assert _relerr(reqs[5][1]["slp"], ref) <= 1e-12


# ---------------------------------------------------------------- Laplace

LAPLACE_FORMS = [("fp64", 0, 0), ("fp64", 2, 0), ("fp64", 4, 0), ("df64", 0, 0), ("df64", 0, 3)]


def _real_densities(rng, n_src, n):
    return [rng.standard_normal(n_src) for _ in range(n)]


LAPLACE_LAYERS = [("slp",), ("slp", "dlp"), ("dlp",)]


def _laplace_ref(g, p, d, layers):
    return oracle.tsqbx_laplace(g, p, d, slp="slp" in layers, dlp="dlp" in layers)


@pytest.mark.parametrize("precision,p_unroll,share", LAPLACE_FORMS)
@pytest.mark.parametrize("p", [0, 1, 2, 9, 20])
@pytest.mark.parametrize("n", [2, 3, 4])
@pytest.mark.parametrize("layers", LAPLACE_LAYERS)
def test_laplace_multi_equals_each_density_alone(pkg, precision, p_unroll, share, p, n, layers):
    rng = np.random.default_rng(1000 + 100 * p + 10 * n + p_unroll + share + 7 * len(layers))
    g = cloud_geometry(rng, n_ctr=10, n_src=180, q_max=0.6, tgt_per_ctr=4, list_frac=0.7)
    dens = _real_densities(rng, g.n_src, n)
    with pkg.Plan(g, "laplace", layers, p=p, precision=precision, max_rhs=4, p_unroll=p_unroll,
                  fp64_share=share) as plan:
        t, outs = plan.submit_multi(dens)
        assert pkg.poll(t, -1)
        for d, o in zip(dens, outs):
            alone = plan.eval(d)
            for l in layers:
                assert np.array_equal(o[l], alone[l]), l
    for d, o in zip(dens, outs):
        ref = _laplace_ref(g, p, d, layers)
        for l in layers:
            assert _relerr(o[l], ref[l]) <= 1e-12, l


@pytest.mark.parametrize("precision,p_unroll,share", LAPLACE_FORMS)
@pytest.mark.parametrize("depth,max_iters,tpc", [(32, 2, 9), (64, 0, 1), (128, 2, 1), (128, 0, 9), (64, 3, 3)])
@pytest.mark.parametrize("layers", [("slp",), ("slp", "dlp")])
def test_laplace_multi_sliced_lists_single_targets(pkg, precision, p_unroll, share, depth, max_iters, tpc, layers):
    """Single-target items (direct loads), multi-target items (staged tiles)
    and sliced lists (partial sums combined per density and layer), at every
    depth."""
    rng = np.random.default_rng(31 + depth + max_iters + tpc + len(layers))
    g = cloud_geometry(rng, n_ctr=8, n_src=500, q_max=0.5, tgt_per_ctr=tpc, list_frac=0.8)
    dens = _real_densities(rng, g.n_src, 3)
    with pkg.Plan(g, "laplace", layers, p=9, precision=precision, max_rhs=3, tile_depth=depth,
                  max_item_iters=max_iters, p_unroll=p_unroll, fp64_share=share) as plan:
        if max_iters:
            assert plan.info()["n_sliced"] > 0
        t, outs = plan.submit_multi(dens, p=7)
        assert pkg.poll(t, -1)
        for d, o in zip(dens, outs):
            alone = plan.eval(d, p=7)
            ref = _laplace_ref(g, 7, d, layers)
            for l in layers:
                assert np.array_equal(o[l], alone[l]), l
                assert _relerr(o[l], ref[l]) <= 1e-12, l


@pytest.mark.parametrize("precision,p_unroll,share", LAPLACE_FORMS)
@pytest.mark.parametrize("layers", LAPLACE_LAYERS)
def test_laplace_multi_four_densities_deepest_tile(pkg, precision, p_unroll, share, layers):
    """The largest staging footprint: four densities at staging depth 128
    (the double-float double layer then fills 48 KB of shared memory per
    block)."""
    rng = np.random.default_rng(53 + p_unroll + share + len(layers))
    g = cloud_geometry(rng, n_ctr=6, n_src=700, q_max=0.5, tgt_per_ctr=6, list_frac=0.9)
    dens = _real_densities(rng, g.n_src, 4)
    with pkg.Plan(g, "laplace", layers, p=9, precision=precision, max_rhs=4, tile_depth=128, p_unroll=p_unroll,
                  fp64_share=share) as plan:
        t, outs = plan.submit_multi(dens)
        assert pkg.poll(t, -1)
        for d, o in zip(dens, outs):
            alone = plan.eval(d)
            ref = _laplace_ref(g, 9, d, layers)
            for l in layers:
                assert np.array_equal(o[l], alone[l]), l
                assert _relerr(o[l], ref[l]) <= 1e-12, l


@pytest.mark.parametrize("precision", ["fp64", "df64"])
@pytest.mark.parametrize("layers", [("slp",), ("slp", "dlp")])
def test_laplace_multi_device_buffers_and_slot_reuse(pkg, precision, layers):
    import torch
    rng = np.random.default_rng(41)
    g = cloud_geometry(rng, n_ctr=8, n_src=300, tgt_per_ctr=5)
    dens = _real_densities(rng, g.n_src, 4)
    with pkg.Plan(g, "laplace", layers, p=8, precision=precision, max_rhs=4, n_slots=2) as plan:
        ddev = [torch.from_numpy(d).cuda() for d in dens]
        t1, o1 = plan.submit_multi(ddev)                       # device in, device out
        t2, o2 = plan.submit_multi(dens[:2])                   # host, on the other slot
        assert pkg.poll(t1, -1) and pkg.poll(t2, -1)
        t3, o3 = plan.submit(dens[3])                          # a single-density call after a multi one
        assert pkg.poll(t3, -1)
        for i in range(4):
            alone = plan.eval(dens[i])
            for l in layers:
                assert o1[i][l].dtype == torch.float64
                assert np.array_equal(o1[i][l].cpu().numpy(), alone[l])
                if i < 2:
                    assert np.array_equal(o2[i][l], alone[l])
        alone = plan.eval(dens[3])
        for l in layers:
            assert np.array_equal(o3[l], alone[l])


def test_laplace_multi_layer_checks(pkg):
    """The double-layer outputs are required exactly when the plan forms the
    double layer; S' and mixed plans take no multi-density evaluation."""
    from paper_1811_01110_gb300 import _lib
    rng = np.random.default_rng(45)
    g = cloud_geometry(rng, n_ctr=4, n_src=60, tgt_per_ctr=2)
    dens = _real_densities(rng, g.n_src, 2)
    for layers in (("slp", "sp"), ("sp",)):
        with pytest.raises(pkg.TsqbxError) as e:
            pkg.Plan(g, "laplace", layers, p=4, max_rhs=2)
        assert e.value.code == _lib.TSQBX_E_UNSUPPORTED
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=4, max_rhs=2) as plan:
        d_addr = (ctypes.c_void_p * 2)(*[d.ctypes.data for d in dens])
        outs = [np.empty(g.n_tgt) for _ in range(2)]
        o_addr = (ctypes.c_void_p * 2)(*[o.ctypes.data for o in outs])
        t = ctypes.c_uint64()
        # tsqbx_submit_multi carries no double-layer outputs
        assert pkg.lib().tsqbx_submit_multi(plan._h, 4, 0.0, 2, d_addr, o_addr, ctypes.byref(t)) == \
            _lib.TSQBX_E_INVAL
        assert pkg.lib().tsqbx_submit_multi_layers(plan._h, 4, 0.0, 2, d_addr, o_addr, None, ctypes.byref(t)) == \
            _lib.TSQBX_E_INVAL
    with pkg.Plan(g, "laplace", ("dlp",), p=4, max_rhs=2) as plan:  # double layer alone: no single-layer outputs
        t, outs = plan.submit_multi(dens)
        assert pkg.poll(t, -1)
        for d, o in zip(dens, outs):
            assert set(o) == {"dlp"}
            assert np.array_equal(o["dlp"], plan.eval(d)["dlp"])


@pytest.mark.parametrize("layers,path", [(("slp",), "df64"), (("slp", "dlp"), "fp64"), (("slp", "dlp"), "df64")])
def test_server_merges_queued_laplace_requests(pkg, layers, path):
    """A burst of Laplace FP64 requests for one geometry and order, served on
    the FP64 or the double-float kernels: queued requests start together in
    multi-density evaluations, and every result equals the request evaluated
    alone on a plan of that precision, bit for bit, and the oracle within
    1e-12."""
    from tsqbx_inputs import configs
    g, _ = configs.sphere(subdiv=2)
    rng = np.random.default_rng(47 + len(layers))
    dens = _real_densities(rng, g.n_src, 16)
    with pkg.Server(hbm_budget=4 << 30, max_inflight=8, laplace_fp64_path=path) as srv:
        gid = srv.add_geometry(g)
        reqs = [srv.submit(gid, d, "laplace", layers, 9, 0.0, "fp64") for d in dens]
        for rid, _ in reqs:
            assert srv.poll(rid, -1)
        st = srv.stats()
    assert st["completed"] == len(dens) and st["failed"] == 0
    assert st["merged"] > 0
    with pkg.Plan(g, "laplace", layers, p=9, precision=path) as alone:
        for d, (rid, outs) in zip(dens, reqs):
            a = alone.eval(d)
            for l in layers:
                assert np.array_equal(outs[l], a[l]), l
    ref = oracle.tsqbx_laplace(g, 9, dens[5], slp=True, dlp="dlp" in layers)
    for l in layers:
        assert _relerr(reqs[5][1][l], ref[l]) <= 1e-12, l
