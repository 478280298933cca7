"""Serving-runtime host logic without a GPU: argument checks, and a request
whose plan cannot be built (no CUDA device here) fails cleanly instead of
hanging the queue."""
import ctypes

import numpy as np
import pytest

from helpers import cloud_geometry


@pytest.fixture(scope="module")
def pkg():
    from paper_1811_01110_gb300 import build
    build.build()
    import paper_1811_01110_gb300 as pkg
    pkg.lib()
    return pkg


def test_server_argument_checks(pkg):
    L = pkg.lib()
    h = ctypes.c_void_p()
    assert L.tsqbx_server_create(0, 0, 4, ctypes.byref(h)) == -1          # zero budget
    assert L.tsqbx_server_create(0, 1 << 20, 0, ctypes.byref(h)) == -1    # no in-flight slots
    assert L.tsqbx_server_create(-1, 1 << 20, 4, ctypes.byref(h)) == -1
    assert L.tsqbx_server_poll(None, ctypes.c_uint64(1), 0) == -1
    assert L.tsqbx_server_set_size_priority(None, 1) == -1
    assert L.tsqbx_server_set_laplace_fp64_path(None, 2) == -1
    assert L.tsqbx_server_create(0, 1 << 20, 4, ctypes.byref(h)) == 0   # worker thread only, no CUDA yet
    try:
        assert L.tsqbx_server_set_laplace_fp64_path(h, 1) == -1          # mixed is not an FP64 path
        assert L.tsqbx_server_set_laplace_fp64_path(h, 2) == 0
        assert L.tsqbx_server_set_laplace_fp64_path(h, 0) == 0
    finally:
        L.tsqbx_server_destroy(h)


def test_request_failure_is_reported_without_gpu(pkg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("this host has a GPU: the failure path needs plan creation to fail")
    rng = np.random.default_rng(3)
    g = cloud_geometry(rng, n_ctr=3, n_src=20)
    with pkg.Server(hbm_budget=1 << 30, max_inflight=2) as srv:
        gid = srv.add_geometry(g)
        with pytest.raises(pkg.TsqbxError):
            srv.submit(gid + 5, np.ones(g.n_src))                      # unknown geometry
        rid, _ = srv.submit(gid, np.ones(g.n_src), "laplace", ("slp",), 3)
        with pytest.raises(pkg.TsqbxError) as ei:
            srv.poll(rid, timeout_us=-1)
        assert ei.value.code in (-4, -3)                                # CUDA unavailable
        st = srv.stats()
        assert st["rejected"] == 1 and st["completed"] == 0 and st["queued"] == 0
