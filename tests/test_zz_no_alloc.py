"""tsqbx_eval_noalloc: the evaluation for callers that cannot call cudaMalloc
(for example a program whose device memory belongs to its own pool).  It takes
device arrays and keeps its scratch in a fixed device array inside the library.

Checked through the C ABI against the plan-based tsqbx_eval on two calls in a
row (the scratch is reused and must not leak between calls), within the FP64
parity tolerance used by the other GPU tests (1e-12 relative).  This file runs
last so that a failure here leaves the rest of the suite already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_01110_gb300 as pkg
    from paper_1811_01110_gb300 import _lib
    pkg.lib()
    return torch, pkg, _lib


def _device_geometry(torch, _lib, g):
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
    src = dev(g.src_xyz, np.float64)
    w = dev(g.src_weight, np.float64)
    nrm = dev(g.src_normal, np.float64)
    ctr = dev(g.ctr_xyz, np.float64)
    tgt = dev(g.tgt_xyz, np.float64)
    tc = dev(g.tgt_center, np.int32)
    cg = dev(g.ctr_group, np.int32)
    grs = dev(g.group_range_start, np.int64)
    rb = dev(g.range_begin, np.int32)
    re = dev(g.range_end, np.int32)
    geo = _lib.tsqbx_geometry(g.n_src, ptr(src, d), ptr(w, d), ptr(nrm, d), g.n_ctr, ptr(ctr, d), None,
                              g.n_tgt, ptr(tgt, d), ptr(tc, i32), g.n_group, ptr(cg, i32),
                              ptr(grs, ctypes.c_int64), ptr(rb, i32), ptr(re, i32))
    return geo, keep


def test_noalloc_matches_plan_eval_twice(env):
    torch, pkg, _lib = env
    from tsqbx_inputs import configs
    g, mu0, _ = configs.torus(48, 18)
    rng = np.random.default_rng(5)
    mus = [mu0, rng.standard_normal(g.n_src)]
    geo, keep = _device_geometry(torch, _lib, g)
    lib = pkg.lib()
    with pkg.Plan(g, "laplace", ("slp", "dlp"), p=9, precision="fp64") as plan:
        for mu in mus:                                   # two calls in a row
            ref = plan.eval(mu)
            dmu = torch.from_numpy(mu).cuda()
            out = {k: torch.full((g.n_tgt,), np.nan, dtype=torch.float64, device="cuda")
                   for k in ("slp", "dlp")}
            rc = lib.tsqbx_eval_noalloc(ctypes.byref(geo), 9, _lib.TSQBX_SLP | _lib.TSQBX_DLP,
                                        ctypes.c_void_p(dmu.data_ptr()),
                                        ctypes.c_void_p(out["slp"].data_ptr()),
                                        ctypes.c_void_p(out["dlp"].data_ptr()), None)
            assert rc == 0, pkg.strerror(rc)
            for layer in ("slp", "dlp"):
                got = out[layer].cpu().numpy()
                err = np.max(np.abs(got - ref[layer])) / np.max(np.abs(ref[layer]))
                assert err <= TOL, (layer, err)


def test_noalloc_rejects_too_many_sources(env):
    torch, pkg, _lib = env
    geo = _lib.tsqbx_geometry()
    geo.n_src = _lib.TSQBX_NOALLOC_MAX_SRC + 1
    rc = pkg.lib().tsqbx_eval_noalloc(ctypes.byref(geo), 3, _lib.TSQBX_SLP, None, None, None, None)
    assert rc == _lib.TSQBX_E_TOO_LARGE
    assert "no-allocation scratch" in pkg.strerror(rc)
