"""ctypes binding of libtsqbx (include/tsqbx.h): argument marshalling only.

Every name mirrors the C ABI.  The shared library is the in-tree
``paper_1811_01110_gb300/libtsqbx.so`` produced by ``build.py``; importing
this module never builds or falls back to anything -- a missing library is an
error.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsqbx.so")

TSQBX_P_MAX = 20
TSQBX_OK, TSQBX_PENDING = 0, 1
TSQBX_E_INVAL, TSQBX_E_DIVERGENT, TSQBX_E_NOMEM, TSQBX_E_CUDA = -1, -2, -3, -4
TSQBX_E_TIMEOUT, TSQBX_E_BUSY, TSQBX_E_NOTFOUND, TSQBX_E_KERNEL = -5, -6, -7, -8
TSQBX_E_UNSUPPORTED = -9
TSQBX_E_TOO_LARGE = -10
TSQBX_NOALLOC_MAX_SRC = 1048544
TSQBX_LAPLACE, TSQBX_HELMHOLTZ = 0, 1
TSQBX_SLP, TSQBX_DLP, TSQBX_SP = 1, 2, 4
TSQBX_FP64, TSQBX_MIXED, TSQBX_DF64 = 0, 1, 2
TSQBX_FLAG_ALLOW_DIVERGENT, TSQBX_FLAG_SKIP_CHECK, TSQBX_FLAG_USE_TUNED = 1, 2, 4
TSQBX_FLAG_CONVENTIONAL_AUTO, TSQBX_FLAG_CONVENTIONAL_ALL = 8, 16
TSQBX_FLAG_SIZE_PRIORITY = 32

_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class tsqbx_geometry(ctypes.Structure):
    _fields_ = [
        ("n_src", ctypes.c_int64), ("src_xyz", _dp), ("src_weight", _dp), ("src_normal", _dp),
        ("n_ctr", ctypes.c_int64), ("ctr_xyz", _dp), ("ctr_radius", _dp),
        ("n_tgt", ctypes.c_int64), ("tgt_xyz", _dp), ("tgt_center", _i32p),
        ("n_group", ctypes.c_int64), ("ctr_group", _i32p), ("group_range_start", _i64p),
        ("range_begin", _i32p), ("range_end", _i32p), ("tgt_normal", _dp),
    ]


class tsqbx_options(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int), ("layers", ctypes.c_uint32), ("p", ctypes.c_int),
        ("k", ctypes.c_double), ("precision", ctypes.c_int), ("device", ctypes.c_int),
        ("flags", ctypes.c_uint32), ("lanes_per_target", ctypes.c_int), ("n_slots", ctypes.c_int),
        ("max_item_iters", ctypes.c_int), ("tile_depth", ctypes.c_int), ("max_rhs", ctypes.c_int),
        ("p_unroll", ctypes.c_int), ("fp64_share", ctypes.c_int),
    ]


class tsqbx_plan_stats(ctypes.Structure):
    _fields_ = [
        ("n_src", ctypes.c_int64), ("n_ctr", ctypes.c_int64), ("n_tgt", ctypes.c_int64),
        ("n_group", ctypes.c_int64), ("n_pairs", ctypes.c_int64), ("n_pair_terms", ctypes.c_int64),
        ("n_items", ctypes.c_int64), ("n_divergent", ctypes.c_int64),
        ("n_coincident", ctypes.c_int64), ("list_entries", ctypes.c_int64),
        ("lane_utilisation", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
        ("n_sliced", ctypes.c_int64), ("launches_per_eval", ctypes.c_int),
        ("n_conv_centers", ctypes.c_int64), ("n_conv_targets", ctypes.c_int64),
        ("n_conv_items", ctypes.c_int64),
    ]


class tsqbx_batch_stats(ctypes.Structure):
    _fields_ = [
        ("n_plans", ctypes.c_int64), ("n_items", ctypes.c_int64), ("n_sliced", ctypes.c_int64),
        ("n_pairs", ctypes.c_int64), ("n_pair_terms", ctypes.c_int64), ("grid_blocks", ctypes.c_int),
        ("graph", ctypes.c_int), ("launches_per_eval", ctypes.c_int), ("device_bytes", ctypes.c_size_t),
    ]


class tsqbx_server_stats(ctypes.Structure):
    _fields_ = [
        ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
        ("max_ms", ctypes.c_double), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
        ("rejected", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
        ("plans_resident", ctypes.c_int64), ("plans_created", ctypes.c_int64),
        ("plans_evicted", ctypes.c_int64), ("resident_bytes", ctypes.c_size_t),
        ("pair_terms_completed", ctypes.c_int64), ("span_s", ctypes.c_double), ("merged", ctypes.c_int64),
    ]


class tsqbx_octree_stats(ctypes.Structure):
    _fields_ = [
        ("n_boxes", ctypes.c_int64), ("n_leaves", ctypes.c_int64), ("max_level", ctypes.c_int64),
        ("n_target_boxes", ctypes.c_int64), ("near_nnz", ctypes.c_int64),
        ("center_source_pairs", ctypes.c_int64), ("build_ms", ctypes.c_double),
        ("upload_ms", ctypes.c_double), ("tree_ms", ctypes.c_double), ("order_ms", ctypes.c_double),
        ("lists_ms", ctypes.c_double), ("download_ms", ctypes.c_double),
    ]


class tsqbx_pipe_peaks(ctypes.Structure):
    _fields_ = [("fp64_tflops", ctypes.c_double), ("fp32_tflops", ctypes.c_double),
                ("fp32x2_tflops", ctypes.c_double), ("sm_count", ctypes.c_int),
                ("ms_fp64", ctypes.c_float), ("ms_fp32", ctypes.c_float), ("ms_fp32x2", ctypes.c_float)]


class tsqbx_tuning(ctypes.Structure):
    _fields_ = [("lanes_per_target", ctypes.c_int), ("max_item_iters", ctypes.c_int),
                ("kernel_ms", ctypes.c_float), ("tile_depth", ctypes.c_int), ("p_unroll", ctypes.c_int),
                ("fp64_share", ctypes.c_int)]


# (name, restype, argtypes) for every entry point declared in include/tsqbx.h
_SIGNATURES = [
    ("tsqbx_plan_create", ctypes.c_int,
     [ctypes.POINTER(tsqbx_geometry), ctypes.POINTER(tsqbx_options), ctypes.POINTER(ctypes.c_void_p)]),
    ("tsqbx_plan_destroy", None, [ctypes.c_void_p]),
    ("tsqbx_plan_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tsqbx_plan_stats)]),
    ("tsqbx_plan_footprint", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("tsqbx_eval", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("tsqbx_eval_async", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("tsqbx_eval_async_pk", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p]),
    ("tsqbx_submit", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.POINTER(ctypes.c_uint64)]),
    ("tsqbx_poll", ctypes.c_int, [ctypes.c_uint64, ctypes.c_int]),
    ("tsqbx_submit_multi", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_uint64)]),
    ("tsqbx_submit_multi_layers", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_uint64)]),
    ("tsqbx_eval_pk", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p]),
    ("tsqbx_submit_pk", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    ("tsqbx_plan_kernel_ms", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("tsqbx_plan_autotune", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(tsqbx_tuning)]),
    ("tsqbx_plan_set_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tsqbx_tuning)]),
    ("tsqbx_plan_get_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tsqbx_tuning)]),
    ("tsqbx_batch_create", ctypes.c_int,
     [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("tsqbx_batch_destroy", None, [ctypes.c_void_p]),
    ("tsqbx_batch_eval_async", ctypes.c_int,
     [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
      ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    ("tsqbx_batch_kernel_ms", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("tsqbx_batch_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tsqbx_batch_stats)]),
    ("tsqbx_server_create", ctypes.c_int,
     [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("tsqbx_server_destroy", None, [ctypes.c_void_p]),
    ("tsqbx_server_add_geometry", ctypes.c_int,
     [ctypes.c_void_p, ctypes.POINTER(tsqbx_geometry), ctypes.POINTER(ctypes.c_int)]),
    ("tsqbx_server_prepare", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(tsqbx_options)]),
    ("tsqbx_server_submit", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(tsqbx_options), ctypes.c_void_p, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    ("tsqbx_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]),
    ("tsqbx_server_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tsqbx_server_stats)]),
    ("tsqbx_server_reset_stats", ctypes.c_int, [ctypes.c_void_p]),
    ("tsqbx_server_set_size_priority", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("tsqbx_server_set_laplace_fp64_path", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("tsqbx_eval_noalloc", ctypes.c_int,
     [ctypes.POINTER(tsqbx_geometry), ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p,
      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("tsqbx_octree_build", ctypes.c_int,
     [ctypes.c_int64, _dp, ctypes.c_int64, _dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
      ctypes.POINTER(ctypes.c_void_p)]),
    ("tsqbx_octree_destroy", None, [ctypes.c_void_p]),
    ("tsqbx_octree_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tsqbx_octree_stats)]),
    ("tsqbx_octree_boxes", ctypes.c_int,
     [ctypes.c_void_p, _i32p, _dp, _dp, _i32p, _i32p, _i32p, _i32p, _i32p]),
    ("tsqbx_octree_order", ctypes.c_int, [ctypes.c_void_p, _i32p, _i32p]),
    ("tsqbx_octree_near", ctypes.c_int, [ctypes.c_void_p, _i64p, _i32p, _i32p]),
    ("tsqbx_measure_pipe_peaks", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(tsqbx_pipe_peaks)]),
    ("tsqbx_last_error", ctypes.c_char_p, []),
    ("tsqbx_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("tsqbx_version", ctypes.c_int, []),
]

_lib = None


def lib():
    """The loaded libtsqbx (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code):
    return lib().tsqbx_strerror(int(code)).decode()


class TsqbxError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = ""
        if code in (TSQBX_E_CUDA, TSQBX_E_NOMEM):
            detail = f" [{lib().tsqbx_last_error().decode()}]"
        super().__init__(f"{where}: {strerror(code)} ({code}){detail}")


def check(code, where):
    if code < 0:
        raise TsqbxError(code, where)
    return code
