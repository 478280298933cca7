"""tsqbx_eval_noalloc: the evaluation for callers that cannot call cudaMalloc
(for example a program whose device memory belongs to its own pool, which a
second allocator would fight).  It takes device arrays and keeps its scratch
in a fixed device array inside the library.

Checked through the C ABI, on two calls in a row (the scratch is shared and
keeps the previous call's contents), against both the FP64 CPU oracle and the
plan-based tsqbx_eval, within the FP64 parity tolerance of the other GPU tests
(1e-12 relative), for orders 0, 1, 2, 9, 20 and every layer mask.  The
device-checked error paths (an index past the sources, a source on its center)
return TSQBX_E_KERNEL without touching memory out of bounds, and the next clean
call succeeds.  This file runs last so that a failure here leaves the rest of
the suite already run.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-12
LAYER_MASKS = {("slp",): 1, ("dlp",): 2, ("slp", "dlp"): 3}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01110_gb300 as pkg
    from paper_1811_01110_gb300 import _lib
    pkg.lib()
    return torch, pkg, _lib


@pytest.fixture(scope="module")
def torus():
    from tsqbx_inputs import configs
    g, mu0, _ = configs.torus(32, 12)
    return g, mu0


def _device_geometry(torch, _lib, g, src_xyz=None, range_end=None):
    """tsqbx_geometry whose pointer fields are device pointers (kept alive in `keep`)."""
    keep = {}

    def dev(a, dtype):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()
        keep[id(t)] = t
        return t

    def ptr(t, ctype):
        return ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(ctype))

    d = ctypes.c_double
    i32 = ctypes.c_int32
    src = dev(g.src_xyz if src_xyz is None else src_xyz, np.float64)
    w = dev(g.src_weight, np.float64)
    nrm = dev(g.src_normal, np.float64)
    ctr = dev(g.ctr_xyz, np.float64)
    tgt = dev(g.tgt_xyz, np.float64)
    tc = dev(g.tgt_center, np.int32)
    cg = dev(g.ctr_group, np.int32)
    grs = dev(g.group_range_start, np.int64)
    rb = dev(g.range_begin, np.int32)
    re = dev(g.range_end if range_end is None else range_end, np.int32)
    geo = _lib.tsqbx_geometry(g.n_src, ptr(src, d), ptr(w, d), ptr(nrm, d), g.n_ctr, ptr(ctr, d), None,
                              g.n_tgt, ptr(tgt, d), ptr(tc, i32), g.n_group, ptr(cg, i32),
                              ptr(grs, ctypes.c_int64), ptr(rb, i32), ptr(re, i32))
    return geo, keep


def _call(torch, pkg, geo, n_tgt, p, mask, mu):
    dmu = torch.from_numpy(np.ascontiguousarray(mu)).cuda()
    out = {k: torch.full((n_tgt,), np.nan, dtype=torch.float64, device="cuda") for k in ("slp", "dlp")}
    rc = pkg.lib().tsqbx_eval_noalloc(ctypes.byref(geo), p, mask, ctypes.c_void_p(dmu.data_ptr()),
                                      ctypes.c_void_p(out["slp"].data_ptr()) if mask & 1 else None,
                                      ctypes.c_void_p(out["dlp"].data_ptr()) if mask & 2 else None, None)
    torch.cuda.synchronize()
    return rc, {k: v.cpu().numpy() for k, v in out.items()}


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("layers", list(LAYER_MASKS))
@pytest.mark.parametrize("p", [0, 1, 2, 9, 20])
def test_noalloc_matches_oracle_and_plan_twice(env, torus, p, layers):
    torch, pkg, _lib = env
    g, mu0 = torus
    rng = np.random.default_rng(5 + p)
    mus = [mu0, rng.standard_normal(g.n_src)]
    geo, keep = _device_geometry(torch, _lib, g)
    # a sample of targets keeps the oracle to a second or two at p = 20
    idx = np.sort(rng.choice(g.n_tgt, 300, replace=False))
    with pkg.Plan(g, "laplace", layers, p=p, precision="fp64") as plan:
        for mu in mus:                                   # two calls in a row
            ref_plan = plan.eval(mu)
            ref = oracle.tsqbx_laplace(g, p, mu, subset=idx, slp="slp" in layers, dlp="dlp" in layers)
            rc, out = _call(torch, pkg, geo, g.n_tgt, p, LAYER_MASKS[layers], mu)
            assert rc == 0, pkg.strerror(rc)
            for layer in layers:
                assert _relerr(out[layer], ref_plan[layer]) <= TOL, ("plan", layer)
                assert _relerr(out[layer][idx], ref[layer]) <= TOL, ("oracle", layer)
            for layer in set(("slp", "dlp")) - set(layers):
                assert np.all(np.isnan(out[layer])), "an output not asked for was written"


def test_noalloc_out_of_range_index_then_clean_call(env, torus):
    """A range end past n_src is skipped on the device and reported as
    TSQBX_E_KERNEL; the next call with valid lists succeeds and is exact."""
    torch, pkg, _lib = env
    g, mu = torus
    bad_end = np.array(g.range_end, np.int32).copy()
    bad_end[len(bad_end) // 2] = g.n_src + 5
    geo_bad, keep_bad = _device_geometry(torch, _lib, g, range_end=bad_end)
    rc, _ = _call(torch, pkg, geo_bad, g.n_tgt, 5, 3, mu)
    assert rc == _lib.TSQBX_E_KERNEL
    geo, keep = _device_geometry(torch, _lib, g)
    rc, out = _call(torch, pkg, geo, g.n_tgt, 5, 3, mu)
    assert rc == 0, pkg.strerror(rc)
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=5) as plan:
        ref = plan.eval(mu)
    for layer in ("slp", "dlp"):
        assert _relerr(out[layer], ref[layer]) <= TOL


def test_noalloc_source_on_center_is_reported(env, torus):
    """A listed source placed exactly on its center (R = 0) has no expansion:
    the pair is skipped and the call returns TSQBX_E_KERNEL, not inf/NaN
    silently; a clean call afterwards succeeds."""
    torch, pkg, _lib = env
    g, mu = torus
    src = np.array(g.src_xyz, np.float64).copy()
    c = int(g.tgt_center[0])
    q = int(g.ctr_group[c])
    s = int(g.range_begin[g.group_range_start[q]])        # first source on that center's list
    src[:, s] = g.ctr_xyz[:, c]
    geo_bad, keep_bad = _device_geometry(torch, _lib, g, src_xyz=src)
    rc, out = _call(torch, pkg, geo_bad, g.n_tgt, 9, 3, mu)
    assert rc == _lib.TSQBX_E_KERNEL
    assert np.all(np.isfinite(out["slp"])) and np.all(np.isfinite(out["dlp"]))
    geo, keep = _device_geometry(torch, _lib, g)
    rc, _ = _call(torch, pkg, geo, g.n_tgt, 9, 3, mu)
    assert rc == 0, pkg.strerror(rc)


def test_noalloc_rejects_too_many_sources(env):
    torch, pkg, _lib = env
    geo = _lib.tsqbx_geometry()
    geo.n_src = _lib.TSQBX_NOALLOC_MAX_SRC + 1
    rc = pkg.lib().tsqbx_eval_noalloc(ctypes.byref(geo), 3, _lib.TSQBX_SLP, None, None, None, None)
    assert rc == _lib.TSQBX_E_TOO_LARGE
    assert "no-allocation scratch" in pkg.strerror(rc)
