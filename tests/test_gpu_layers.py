"""GPU parity for the derivative layers: S' (target-normal derivative of the
single layer, Laplace and Helmholtz) and the Helmholtz double layer, through
the C ABI, against the FP64 CPU oracle (Appendix A).

Tolerances (max-norm relative, per layer): FP64 and df64 1e-12; mixed 1e-6
for every layer, S' included (measured on a GB300 over every test case below:
at most 5.5e-7 for S', 9.4e-7 for the double layer).
"""
import numpy as np
import pytest

import oracle
from helpers import cloud_geometry
from tsqbx_inputs import configs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6, "df64": 1e-12}
TOL_SP = {"fp64": 1e-12, "mixed": 1e-6, "df64": 1e-12}


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


def tol(layer, precision):
    return (TOL_SP if layer == "sp" else TOL)[precision]


def check_laplace(pkg, g, mu, p, precision, layers, **kw):
    ref = oracle.tsqbx_laplace(g, p, mu, slp=True, dlp="dlp" in layers, sp="sp" in layers)
    with pkg.Plan(g, "laplace", layers, p=p, precision=precision, **kw) as plan:
        out = plan.eval(mu)
    for layer in layers:
        e = relerr(out[layer], ref[layer])
        assert e <= tol(layer, precision), (layer, precision, p, e)
    return out


def check_helmholtz(pkg, g, mu, p, k, layers, **kw):
    ref = oracle.tsqbx_helmholtz(g, p, k, mu, slp=True, dlp="dlp" in layers, sp="sp" in layers)
    with pkg.Plan(g, "helmholtz", layers, p=p, k=k, **kw) as plan:
        out = plan.eval(mu)
    for layer in layers:
        e = relerr(out[layer], ref[layer])
        assert e <= 1e-12, (layer, p, k, e)
    return out


# ------------------------------------------------------------------ Laplace S'

@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("p", list(range(0, 21)))
def test_laplace_sp_every_order(pkg, precision, p):
    rng = np.random.default_rng(300 + p)
    g = cloud_geometry(rng, n_ctr=12, n_src=150, q_max=0.6, tgt_per_ctr=3, list_frac=0.7)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, p, precision, ("slp", "dlp", "sp"))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("layers", [("sp",), ("slp", "sp"), ("dlp", "sp")])
def test_laplace_sp_layer_subsets(pkg, precision, layers):
    rng = np.random.default_rng(41)
    g = cloud_geometry(rng, n_ctr=9, n_src=200, q_max=0.5, tgt_per_ctr=6, list_frac=0.8)
    mu = rng.standard_normal(g.n_src)
    out = check_laplace(pkg, g, mu, 8, precision, layers)
    assert set(out) == set(layers)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
def test_laplace_sp_target_on_center(pkg, precision):
    """t = c (rho = 0): only the n = 1 term of S' survives, (d.n_t)/R^3."""
    rng = np.random.default_rng(43)
    g = cloud_geometry(rng, n_ctr=6, n_src=120, tgt_per_ctr=4, rho_zero=True)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, 9, precision, ("slp", "dlp", "sp"))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("lanes,max_iters", [(1, 0), (3, 0), (8, 2), (32, 0), (0, 1), (0, 7)])
def test_laplace_sp_lanes_and_slices(pkg, precision, lanes, max_iters):
    """Ragged items (forced lane counts) and sliced lists (partials combined)."""
    rng = np.random.default_rng(47)
    g = cloud_geometry(rng, n_ctr=6, n_src=300, q_max=0.5, tgt_per_ctr=23, list_frac=0.9)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, 7, precision, ("slp", "sp"), lanes_per_target=lanes,
                  max_item_iters=max_iters)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("max_iters", [0, 3])
def test_laplace_sp_single_target_groups(pkg, precision, max_iters):
    """One target per group: the direct-load path."""
    rng = np.random.default_rng(53)
    g = cloud_geometry(rng, n_ctr=40, n_src=500, q_max=0.6, tgt_per_ctr=1, list_frac=0.5)
    mu = rng.standard_normal(g.n_src)
    check_laplace(pkg, g, mu, 9, precision, ("slp", "dlp", "sp"), max_item_iters=max_iters)


def test_laplace_sp_torus_sampled_targets(pkg):
    """Torus 256 x 96 with octree lists at p = 9, sampled targets."""
    g, mu, _ = configs.torus()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(g.n_tgt, 400, replace=False))
    ref = oracle.tsqbx_laplace(g, 9, mu, subset=idx, slp=True, sp=True)
    for precision in ("fp64", "mixed", "df64"):
        with pkg.Plan(g, "laplace", ("slp", "sp"), p=9, precision=precision) as plan:
            out = plan.eval(mu)
        for layer in ("slp", "sp"):
            e = relerr(out[layer][idx], ref[layer])
            assert e <= tol(layer, precision), (precision, layer, e)


def test_sp_only_when_an_output_is_given(pkg):
    """tsqbx_eval on an S' plan forms the single/double layers only; the
    per-call tsqbx_eval_pk with an S' output forms all three, and the shared
    layers are bit-identical between the two calls."""
    from paper_1811_01110_gb300 import _lib
    import ctypes
    rng = np.random.default_rng(59)
    g = cloud_geometry(rng, n_ctr=8, n_src=150, tgt_per_ctr=5)
    mu = rng.standard_normal(g.n_src)
    with pkg.Plan(g, "laplace", ("slp", "dlp", "sp"), p=6) as plan:
        full = plan.eval(mu)
        a = np.full(g.n_tgt, 7.0)
        b = np.full(g.n_tgt, 7.0)
        rc = pkg.lib().tsqbx_eval(plan._h, ctypes.c_void_p(np.ascontiguousarray(mu).ctypes.data),
                                  ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data))
        assert rc == _lib.TSQBX_OK
    assert np.array_equal(a, full["slp"]) and np.array_equal(b, full["dlp"])


def test_sp_submit_and_device_outputs(pkg):
    import torch
    rng = np.random.default_rng(61)
    g = cloud_geometry(rng, n_ctr=8, n_src=150, tgt_per_ctr=5)
    mu = rng.standard_normal(g.n_src)
    with pkg.Plan(g, "laplace", ("slp", "sp"), p=6, n_slots=2) as plan:
        host = plan.eval(mu)
        dmu = torch.from_numpy(mu).cuda()
        dev = plan.eval(dmu)
        t, outs = plan.submit(mu)
        assert pkg.poll(t, -1)
        asy = {l: torch.full((g.n_tgt,), 7.0, dtype=torch.float64, device="cuda") for l in ("slp", "sp")}
        plan.eval_async(dmu, asy, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        asy_p4 = {l: torch.empty(g.n_tgt, dtype=torch.float64, device="cuda") for l in ("slp", "sp")}
        plan.eval_async(dmu, asy_p4, stream=torch.cuda.current_stream(), p=4)
        torch.cuda.synchronize()
    assert np.array_equal(dev["sp"].cpu().numpy(), host["sp"])
    assert np.array_equal(outs["sp"], host["sp"])
    assert np.array_equal(asy["sp"].cpu().numpy(), host["sp"])
    ref4 = oracle.tsqbx_laplace(g, 4, mu, slp=True, sp=True)
    for layer in ("slp", "sp"):
        assert relerr(asy_p4[layer].cpu().numpy(), ref4[layer]) <= 1e-12


# ------------------------------------------------- Helmholtz double layer, S'

@pytest.mark.parametrize("p,k", [(0, 1.0), (1, 2.0), (4, 5.0), (9, 0.5), (12, 10.0), (16, 3.0), (20, 3.0)])
def test_helmholtz_all_layers(pkg, p, k):
    rng = np.random.default_rng(p + 71)
    g = cloud_geometry(rng, n_ctr=10, n_src=120, q_max=0.6, tgt_per_ctr=3, rho_zero=True)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    check_helmholtz(pkg, g, mu, p, k, ("slp", "dlp", "sp"))


@pytest.mark.parametrize("layers", [("dlp",), ("sp",), ("slp", "dlp"), ("dlp", "sp")])
def test_helmholtz_layer_subsets(pkg, layers):
    rng = np.random.default_rng(73)
    g = cloud_geometry(rng, n_ctr=8, n_src=150, q_max=0.5, tgt_per_ctr=4)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    check_helmholtz(pkg, g, mu, 8, 4.0, layers)


@pytest.mark.parametrize("max_iters,lanes", [(1, 0), (5, 0), (0, 3), (2, 7)])
def test_helmholtz_derivatives_sliced(pkg, max_iters, lanes):
    rng = np.random.default_rng(79)
    g = cloud_geometry(rng, n_ctr=5, n_src=300, q_max=0.5, tgt_per_ctr=7, list_frac=0.9)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    check_helmholtz(pkg, g, mu, 8, 4.0, ("slp", "dlp", "sp"), max_item_iters=max_iters,
                    lanes_per_target=lanes)


def test_helmholtz_dlp_small_torus(pkg):
    """The combined-field operator's parts on a torus with octree lists."""
    g, mu, _ = configs.torus_helmholtz(40, 16, k=10.0)
    check_helmholtz(pkg, g, mu, 12, 10.0, ("slp", "dlp", "sp"))


def test_helmholtz_per_call_order_and_wavenumber(pkg):
    rng = np.random.default_rng(83)
    g = cloud_geometry(rng, n_ctr=6, n_src=100, tgt_per_ctr=3)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    with pkg.Plan(g, "helmholtz", ("dlp", "sp"), p=4, k=1.0) as plan:
        for p, k in ((3, 2.0), (11, 7.5)):
            out = plan.eval(mu, p=p, k=k)
            ref = oracle.tsqbx_helmholtz(g, p, k, mu, slp=False, dlp=True, sp=True)
            for layer in ("dlp", "sp"):
                assert relerr(out[layer], ref[layer]) <= 1e-12, (p, k, layer)


def test_server_sp_request(pkg):
    rng = np.random.default_rng(89)
    g = cloud_geometry(rng, n_ctr=6, n_src=100, tgt_per_ctr=3)
    mu = rng.standard_normal(g.n_src)
    ref = oracle.tsqbx_laplace(g, 5, mu, slp=True, sp=True)
    with pkg.Server(hbm_budget=1 << 30) as srv:
        gid = srv.add_geometry(g)
        rid, outs = srv.submit(gid, mu, layers=("slp", "sp"), p=5)
        assert srv.poll(rid, -1)
    for layer in ("slp", "sp"):
        assert relerr(outs[layer], ref[layer]) <= 1e-12
