"""The C ABI library without a GPU: it loads, exports every entry point that
include/tsqbx.h declares, and rejects invalid input on the host before any
CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsqbx.h")


@pytest.fixture(scope="module")
def L():
    from paper_1811_01110_gb300 import build
    build.build()
    import paper_1811_01110_gb300 as pkg
    return pkg.lib()


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"TSQBX_API\s+[\w\s\*]+?\b(tsqbx_\w+)\s*\(", text)


def test_header_declares_the_entry_points():
    names = set(declared_functions())
    assert {"tsqbx_plan_create", "tsqbx_eval", "tsqbx_submit", "tsqbx_poll",
            "tsqbx_plan_destroy", "tsqbx_strerror"} <= names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name
    binding = {n for n, _, _ in __import__("paper_1811_01110_gb300._lib", fromlist=["x"])._SIGNATURES}
    assert binding == set(declared_functions())


def test_strerror_and_version(L):
    import paper_1811_01110_gb300 as pkg
    assert L.tsqbx_version() >= 10500          # 1.5: tsqbx_submit_multi_layers
    for code in range(-10, 2):
        assert pkg.strerror(code) != "unknown status"
    assert pkg.strerror(-100) == "unknown status"


def test_poll_unknown_ticket(L):
    assert L.tsqbx_poll(ctypes.c_uint64(123456789), 0) == -7


def _tiny(rng=np.random.default_rng(0)):
    from helpers import cloud_geometry
    return cloud_geometry(rng, n_ctr=3, n_src=10)


def _create(g, **kw):
    import paper_1811_01110_gb300 as pkg
    try:
        pkg.Plan(g, **kw)
    except pkg.TsqbxError as e:
        return e.code
    return 0


@pytest.mark.parametrize("mutate,code", [
    (lambda g: setattr(g, "tgt_center", np.full_like(g.tgt_center, 99)), -1),
    (lambda g: setattr(g, "range_end", g.range_end + 1000), -1),
    (lambda g: setattr(g, "range_begin", g.range_end + 1), -1),
    (lambda g: setattr(g, "group_range_start", g.group_range_start[::-1].copy()), -1),
    (lambda g: setattr(g, "ctr_group", np.full_like(g.ctr_group, -1)), -1),
    (lambda g: g.src_xyz.__setitem__((0, 0), np.nan), -1),
    (lambda g: g.tgt_xyz.__setitem__((2, 1), np.inf), -1),
    (lambda g: g.ctr_xyz.__setitem__((1, 0), np.nan), -1),
    (lambda g: g.src_weight.__setitem__(3, np.nan), -1),
    (lambda g: setattr(g, "group_range_start", g.group_range_start + 1), -1),
    (lambda g: setattr(g, "ctr_group", np.full_like(g.ctr_group, 99)), -1),
    (lambda g: setattr(g, "range_begin", np.full_like(g.range_begin, -1)), -1),
])
def test_invalid_geometry_rejected_on_host(L, mutate, code):
    g = _tiny()
    mutate(g)
    assert _create(g) == code


def test_nonfinite_normal_rejected_only_with_the_double_layer(L):
    g = _tiny()
    g.src_normal = g.src_normal.copy()
    g.src_normal[0, 2] = np.nan
    assert _create(g, layers=("slp", "dlp")) == -1
    assert _create(g, kernel="helmholtz", k=2.0, layers=("dlp",)) == -1


def test_more_invalid_options_rejected_on_host(L):
    g = _tiny()
    assert _create(g, n_slots=65) == -1
    assert _create(g, max_item_iters=-1) == -1
    assert _create(g, lanes_per_target=-1) == -1
    assert _create(g, kernel="helmholtz", k=float("inf")) == -1
    assert _create(g, kernel="helmholtz", k=float("nan")) == -1
    assert _create(g, kernel="helmholtz", k=-1.0) == -1
    for depth in (-64, 16, 48, 96, 256):                  # staging depth: 0, 32, 64 or 128
        assert _create(g, tile_depth=depth) == -1
    for rhs in (-1, 5):                                    # densities per evaluation: 0..4
        assert _create(g, kernel="helmholtz", k=1.0, max_rhs=rhs) == -1
    # several densities: the Helmholtz single layer, the Laplace single and/or
    # double layer in FP64 or df64 (no S', no mixed).  The accepted
    # combinations pass validation and stop only at the missing device
    # (TSQBX_E_CUDA, -4, on a machine without a GPU).
    for kw in (dict(max_rhs=2), dict(layers=("slp", "dlp"), max_rhs=3), dict(layers=("dlp",), max_rhs=4),
               dict(precision="df64", layers=("slp", "dlp"), max_rhs=4),
               dict(kernel="helmholtz", k=1.0, max_rhs=4)):
        assert _create(g, **kw) not in (-1, -9), kw
    assert _create(g, precision="mixed", max_rhs=2) == -9
    assert _create(g, precision="df64", layers=("slp", "sp"), max_rhs=2) == -9
    assert _create(g, layers=("slp", "dlp", "sp"), max_rhs=2) == -9
    assert _create(g, kernel="helmholtz", k=1.0, layers=("slp", "dlp"), max_rhs=2) == -9
    for unroll in (-1, 3, 8):                              # order-loop forms: 0, 1, 2 or 4
        assert _create(g, p_unroll=unroll) == -1
    # the runtime-order kernels exist for Laplace FP64 and mixed only
    assert _create(g, kernel="helmholtz", k=1.0, p_unroll=2) == -9
    assert _create(g, precision="df64", p_unroll=2) == -9
    for share in (-1, 21):                                 # FP64 share of a df64 launch: 0..20
        assert _create(g, precision="df64", fp64_share=share) == -1
    assert _create(g, fp64_share=2) == -9                  # FP64 items inside df64 plans only
    assert _create(g, precision="mixed", fp64_share=2) == -9


def test_invalid_options_rejected_on_host(L):
    g = _tiny()
    assert _create(g, p=-1) == -1
    assert _create(g, p=21) == -1
    assert _create(g, kernel="helmholtz", k=0.0) == -1
    assert _create(g, kernel="helmholtz", k=1.0, precision="mixed") == -9
    assert _create(g, lanes_per_target=33) == -1
    g.src_normal = None
    assert _create(g, layers=("slp", "dlp")) == -1
    assert _create(g, kernel="helmholtz", k=1.0, layers=("dlp",)) == -1


def test_sp_needs_finite_target_normals(L):
    g = _tiny()
    g.tgt_normal = None
    assert _create(g, layers=("slp", "sp")) == -1
    assert _create(g, kernel="helmholtz", k=1.0, layers=("sp",)) == -1
    g = _tiny()
    g.tgt_normal[1, 0] = np.inf
    assert _create(g, layers=("sp",)) == -1


def test_unknown_layer_bits_rejected(L):
    import paper_1811_01110_gb300 as pkg
    from paper_1811_01110_gb300 import _lib
    g = _tiny()
    geo, keep = pkg.marshal_geometry(g)
    for mask in (0, 8, 1 | 16):
        opt = pkg.make_options()
        opt.layers = mask
        h = ctypes.c_void_p()
        assert L.tsqbx_plan_create(ctypes.byref(geo), ctypes.byref(opt), ctypes.byref(h)) == _lib.TSQBX_E_INVAL


def test_conventional_needs_fp64_within_its_orders(L):
    """The conventional path runs in FP64 only, for Laplace p <= 20 and
    Helmholtz p <= 12; other requests are refused on the host."""
    g = _tiny()
    assert _create(g, conventional="all", precision="mixed") == -9
    assert _create(g, conventional="auto", precision="df64") == -9
    assert _create(g, kernel="helmholtz", k=1.0, conventional="all", p=13) == -9


def test_octree_inputs_rejected_on_host(L):
    import paper_1811_01110_gb300 as pkg
    rng = np.random.default_rng(1)
    src, ctr, rad = rng.uniform(-1, 1, (20, 3)), rng.uniform(-1, 1, (5, 3)), np.full(5, 0.01)
    for kw, args in ((dict(n_max=0), (src, ctr, rad)), (dict(t_f=-1.0), (src, ctr, rad)),
                     (dict(), (np.full((20, 3), np.nan), ctr, rad)), (dict(), (src, ctr, -rad))):
        with pytest.raises(pkg.TsqbxError) as ei:
            pkg.Octree(*args, **kw)
        assert ei.value.code == -1


def test_null_handles_rejected_on_host(L):
    """Every entry point that takes a plan or batch handle rejects NULL (and
    NULL outputs) with TSQBX_E_INVAL before any CUDA call; destroy accepts NULL."""
    from paper_1811_01110_gb300 import _lib
    inval = _lib.TSQBX_E_INVAL
    ms = ctypes.c_float()
    nbytes = ctypes.c_size_t()
    assert L.tsqbx_plan_info(None, ctypes.byref(_lib.tsqbx_plan_stats())) == inval
    assert L.tsqbx_plan_footprint(None, ctypes.byref(nbytes)) == inval
    assert L.tsqbx_plan_kernel_ms(None, ctypes.byref(ms)) == inval
    assert L.tsqbx_plan_get_tuning(None, ctypes.byref(_lib.tsqbx_tuning())) == inval
    assert L.tsqbx_plan_set_tuning(None, ctypes.byref(_lib.tsqbx_tuning())) == inval
    assert L.tsqbx_plan_autotune(None, None, 3, None) == inval
    L.tsqbx_plan_destroy(None)
    # batches
    out = ctypes.c_void_p()
    assert L.tsqbx_batch_create(None, 1, 1, ctypes.byref(out)) == inval
    plans = (ctypes.c_void_p * 2)(None, None)
    assert L.tsqbx_batch_create(plans, 2, 1, ctypes.byref(out)) == inval
    assert L.tsqbx_batch_create(plans, 0, 1, ctypes.byref(out)) == inval
    assert L.tsqbx_batch_create(plans, 2, 1, None) == inval
    assert L.tsqbx_batch_eval_async(None, None, None, None, None) == inval
    assert L.tsqbx_batch_kernel_ms(None, ctypes.byref(ms)) == inval
    assert L.tsqbx_batch_info(None, ctypes.byref(_lib.tsqbx_batch_stats())) == inval
    L.tsqbx_batch_destroy(None)


def test_noalloc_arguments_rejected_on_host(L):
    """tsqbx_eval_noalloc checks its counts, order, layer mask and pointers on
    the host; more sources than its scratch holds is TSQBX_E_TOO_LARGE."""
    from paper_1811_01110_gb300 import _lib
    inval = _lib.TSQBX_E_INVAL
    fake = ctypes.c_void_p(16)             # never dereferenced: every call below returns first
    geo = _lib.tsqbx_geometry()
    geo.n_src, geo.n_ctr, geo.n_tgt, geo.n_group = 10, 1, 1, 1
    assert L.tsqbx_eval_noalloc(None, 3, 1, fake, fake, None, None) == inval
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), -1, 1, fake, fake, None, None) == inval
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 21, 1, fake, fake, None, None) == inval
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 0, fake, fake, None, None) == inval
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 4, fake, fake, fake, None) == inval   # S' not offered
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 1, fake, fake, None, None) == inval   # NULL arrays
    # every array present except the range arrays, with n_group > 0
    dp = ctypes.cast(fake, ctypes.POINTER(ctypes.c_double))
    ip = ctypes.cast(fake, ctypes.POINTER(ctypes.c_int32))
    geo.src_xyz = geo.src_weight = geo.ctr_xyz = geo.tgt_xyz = dp
    geo.tgt_center = geo.ctr_group = ip
    geo.group_range_start = ctypes.cast(fake, ctypes.POINTER(ctypes.c_int64))
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 1, fake, fake, None, None) == inval   # NULL ranges
    geo.range_begin = ip
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 1, fake, fake, None, None) == inval   # NULL range_end
    geo.range_begin, geo.range_end = None, ip
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 1, fake, fake, None, None) == inval   # NULL range_begin
    geo.n_src = 1048544 + 1
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 1, fake, fake, None, None) == _lib.TSQBX_E_TOO_LARGE
    geo.n_src = -1
    assert L.tsqbx_eval_noalloc(ctypes.byref(geo), 3, 1, fake, fake, None, None) == inval


def test_submit_multi_rejects_null_on_host(L):
    from paper_1811_01110_gb300 import _lib
    t = ctypes.c_uint64()
    assert L.tsqbx_submit_multi(None, 3, 1.0, 2, None, None, ctypes.byref(t)) == _lib.TSQBX_E_INVAL
    assert L.tsqbx_submit_multi_layers(None, 3, 1.0, 2, None, None, None, ctypes.byref(t)) == _lib.TSQBX_E_INVAL


def test_pipe_peak_probe_rejects_null_on_host(L):
    """tsqbx_measure_pipe_peaks checks its output pointer before any CUDA call."""
    from paper_1811_01110_gb300 import _lib
    assert L.tsqbx_measure_pipe_peaks(0, None) == _lib.TSQBX_E_INVAL
