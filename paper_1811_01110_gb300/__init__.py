"""paper_1811_01110_gb300 -- the near-field TSQBX step of GIGAQBX on GB300.

Thin Python binding over the C ABI of ``libtsqbx`` (include/tsqbx.h).  All
arithmetic runs in the library's CUDA kernels; this module only marshals
arguments (numpy arrays for host memory, torch CUDA tensors for device
memory) and raises on error codes.

    plan = Plan(geometry, kernel="laplace", layers=("slp", "dlp"), p=9,
                precision="fp64")
    u = plan.eval(density)             # {'slp': ndarray, 'dlp': ndarray}

Layers: "slp" (single layer), "dlp" (double layer, source-normal
derivative), "sp" (S', the target-normal derivative of the single layer;
needs geometry.tgt_normal).
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import TsqbxError, check, lib, strerror  # noqa: F401

_KERNELS = {"laplace": _lib.TSQBX_LAPLACE, "helmholtz": _lib.TSQBX_HELMHOLTZ}
_PRECISIONS = {"fp64": _lib.TSQBX_FP64, "mixed": _lib.TSQBX_MIXED, "df64": _lib.TSQBX_DF64}
_LAYERS = {"slp": _lib.TSQBX_SLP, "dlp": _lib.TSQBX_DLP, "sp": _lib.TSQBX_SP}


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


def _is_torch(x):
    return hasattr(x, "data_ptr") and hasattr(x, "is_cuda")


def _addr(x, nbytes, what):
    """Raw address of a numpy array or torch tensor holding at least nbytes."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if x.numel() * x.element_size() < nbytes:
            raise ValueError(f"{what} is too small")
        return ctypes.c_void_p(x.data_ptr())
    if not isinstance(x, np.ndarray) or not x.flags.c_contiguous:
        raise ValueError(f"{what} must be a C-contiguous numpy array or torch tensor")
    if x.nbytes < nbytes:
        raise ValueError(f"{what} is too small")
    return ctypes.c_void_p(x.ctypes.data)


def marshal_geometry(g, with_normals=True, with_tgt_normals=False):
    """tsqbx_geometry view of a geometry object (host numpy arrays); returns
    (struct, keep) where keep holds the contiguous copies alive."""
    f64 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    keep = dict(src_xyz=f64(g.src_xyz), src_weight=f64(g.src_weight),
                src_normal=f64(g.src_normal) if with_normals else None,
                ctr_xyz=f64(g.ctr_xyz), ctr_radius=f64(getattr(g, "ctr_radius", None)),
                tgt_xyz=f64(g.tgt_xyz), tgt_center=i32(g.tgt_center), ctr_group=i32(g.ctr_group),
                group_range_start=np.ascontiguousarray(g.group_range_start, dtype=np.int64),
                range_begin=i32(g.range_begin), range_end=i32(g.range_end),
                tgt_normal=f64(getattr(g, "tgt_normal", None)) if with_tgt_normals else None)
    n_tgt = int(keep["tgt_xyz"].shape[1]) if keep["tgt_xyz"].ndim == 2 else 0
    geo = _lib.tsqbx_geometry(
        int(keep["src_weight"].shape[0]), _ptr(keep["src_xyz"], ctypes.c_double),
        _ptr(keep["src_weight"], ctypes.c_double), _ptr(keep["src_normal"], ctypes.c_double),
        int(keep["ctr_xyz"].shape[1]), _ptr(keep["ctr_xyz"], ctypes.c_double),
        _ptr(keep["ctr_radius"], ctypes.c_double),
        n_tgt, _ptr(keep["tgt_xyz"], ctypes.c_double), _ptr(keep["tgt_center"], ctypes.c_int32),
        int(keep["group_range_start"].shape[0] - 1), _ptr(keep["ctr_group"], ctypes.c_int32),
        _ptr(keep["group_range_start"], ctypes.c_int64),
        _ptr(keep["range_begin"], ctypes.c_int32), _ptr(keep["range_end"], ctypes.c_int32),
        _ptr(keep["tgt_normal"], ctypes.c_double))
    return geo, keep


def make_options(kernel="laplace", layers=("slp",), p=5, k=0.0, precision="fp64", device=0, flags=0,
                 lanes_per_target=0, n_slots=2, max_item_iters=0, tile_depth=0, max_rhs=0, p_unroll=0,
                 fp64_share=0):
    mask = 0
    for name in layers:
        mask |= _LAYERS[name]
    return _lib.tsqbx_options(_KERNELS[kernel], mask, int(p), float(k), _PRECISIONS[precision],
                              int(device), int(flags), int(lanes_per_target), int(n_slots),
                              int(max_item_iters), int(tile_depth), int(max_rhs), int(p_unroll),
                              int(fp64_share))


class Plan:
    """A device-resident TSQBX evaluation plan (tsqbx_plan_create)."""

    def __init__(self, geometry, kernel="laplace", layers=("slp",), p=5, k=0.0,
                 precision="fp64", device=0, allow_divergent=False, skip_check=False,
                 lanes_per_target=0, n_slots=2, max_item_iters=0, use_tuned=False,
                 conventional="off", size_priority=False, tile_depth=0, max_rhs=0, p_unroll=0,
                 fp64_share=0):
        """conventional: "off" (target-specific expansions only), "auto"
        (conventional QBX for the centers the cost model finds cheaper) or
        "all" (conventional QBX for every center).  size_priority: stream
        priority from the plan's work (TSQBX_FLAG_SIZE_PRIORITY).  tile_depth:
        sources staged per warp tile (32, 64 or 128; 0 = 64).  max_rhs:
        densities one submit_multi may carry (the Helmholtz single layer; the
        Laplace single and/or double layer in FP64 or df64).
        p_unroll: 0 = per-order kernels with the recurrences fully unrolled;
        1, 2 or 4 = the runtime-order kernel, its loop over n unrolled by that
        factor (Laplace FP64 and mixed).  fp64_share: df64 plans, the
        twentieths of the work items that run in native FP64 on the FP64 pipe
        beside the double-float items (0..20)."""
        self.kernel = kernel
        self.layers = tuple(layers)
        self.p = int(p)
        self.k = float(k)
        self.complex = kernel == "helmholtz"
        geo, keep = marshal_geometry(geometry, with_normals="dlp" in self.layers,
                                     with_tgt_normals="sp" in self.layers)
        self.n_src, self.n_tgt = int(geo.n_src), int(geo.n_tgt)
        flags = (_lib.TSQBX_FLAG_ALLOW_DIVERGENT if allow_divergent else 0) | \
                (_lib.TSQBX_FLAG_SKIP_CHECK if skip_check else 0) | \
                (_lib.TSQBX_FLAG_USE_TUNED if use_tuned else 0) | \
                {"off": 0, "auto": _lib.TSQBX_FLAG_CONVENTIONAL_AUTO,
                 "all": _lib.TSQBX_FLAG_CONVENTIONAL_ALL}[conventional] | \
                (_lib.TSQBX_FLAG_SIZE_PRIORITY if size_priority else 0)
        opt = make_options(kernel, self.layers, self.p, k, precision, device, flags,
                           lanes_per_target, n_slots, max_item_iters, tile_depth, max_rhs, p_unroll,
                           fp64_share)
        h = ctypes.c_void_p()
        check(lib().tsqbx_plan_create(ctypes.byref(geo), ctypes.byref(opt), ctypes.byref(h)),
              "tsqbx_plan_create")
        self._h = h
        self.width = 2 if self.complex else 1

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tsqbx_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- queries
    def info(self):
        st = _lib.tsqbx_plan_stats()
        check(lib().tsqbx_plan_info(self._h, ctypes.byref(st)), "tsqbx_plan_info")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def footprint(self):
        b = ctypes.c_size_t()
        check(lib().tsqbx_plan_footprint(self._h, ctypes.byref(b)), "tsqbx_plan_footprint")
        return int(b.value)

    def kernel_ms(self):
        """Event-timed duration of the last expansion kernel (tsqbx_plan_kernel_ms)."""
        ms = ctypes.c_float()
        check(lib().tsqbx_plan_kernel_ms(self._h, ctypes.byref(ms)), "tsqbx_plan_kernel_ms")
        return float(ms.value)

    # -- tuning
    def autotune(self, density, repeats=3):
        """tsqbx_plan_autotune on a device density; returns the chosen tuning."""
        t = _lib.tsqbx_tuning()
        check(lib().tsqbx_plan_autotune(self._h, self._density_addr(density), int(repeats),
                                        ctypes.byref(t)), "tsqbx_plan_autotune")
        return {"lanes_per_target": t.lanes_per_target, "max_item_iters": t.max_item_iters,
                "tile_depth": t.tile_depth, "p_unroll": t.p_unroll, "fp64_share": t.fp64_share,
                "kernel_ms": t.kernel_ms}

    def get_tuning(self):
        t = _lib.tsqbx_tuning()
        check(lib().tsqbx_plan_get_tuning(self._h, ctypes.byref(t)), "tsqbx_plan_get_tuning")
        return {"lanes_per_target": t.lanes_per_target, "max_item_iters": t.max_item_iters,
                "tile_depth": t.tile_depth, "p_unroll": t.p_unroll, "fp64_share": t.fp64_share}

    def set_tuning(self, lanes_per_target=0, max_item_iters=0, tile_depth=0, p_unroll=0, fp64_share=0):
        t = _lib.tsqbx_tuning(int(lanes_per_target), int(max_item_iters), 0.0, int(tile_depth), int(p_unroll),
                              int(fp64_share))
        check(lib().tsqbx_plan_set_tuning(self._h, ctypes.byref(t)), "tsqbx_plan_set_tuning")

    # -- evaluation
    def _density_addr(self, density):
        if _is_torch(density):
            return _addr(density, self.n_src * 8 * self.width, "density")
        dt = np.complex128 if self.complex else np.float64
        d = np.ascontiguousarray(density, dtype=dt)
        self._keep_density = d
        return _addr(d, self.n_src * 8 * self.width, "density")

    def _alloc_out(self, like_torch):
        outs = {}
        for name in self.layers:
            if like_torch is not None:
                import torch
                dt = torch.complex128 if self.complex else torch.float64
                outs[name] = torch.empty(self.n_tgt, dtype=dt, device=like_torch.device)
            else:
                outs[name] = np.empty(self.n_tgt, dtype=np.complex128 if self.complex else np.float64)
        return outs

    def _out_addrs(self, outs):
        nb = self.n_tgt * 8 * self.width
        return (_addr(outs.get("slp"), nb, "out_slp"), _addr(outs.get("dlp"), nb, "out_dlp"),
                _addr(outs.get("sp"), nb, "out_sp"))

    def eval(self, density, out=None, p=None, k=None):
        """Blocking evaluation (tsqbx_eval; tsqbx_eval_pk when p or k is given
        or the plan forms S').  density: numpy (host) or torch CUDA tensor;
        returns a dict of outputs of the same kind."""
        like = density if _is_torch(density) and density.is_cuda else None
        outs = out if out is not None else self._alloc_out(like)
        a_slp, a_dlp, a_sp = self._out_addrs(outs)
        d = self._density_addr(density)
        if p is None and k is None and a_sp is None:
            check(lib().tsqbx_eval(self._h, d, a_slp, a_dlp), "tsqbx_eval")
        else:
            pp = self.p if p is None else int(p)
            kk = self.k if k is None else float(k)
            check(lib().tsqbx_eval_pk(self._h, pp, kk, d, a_slp, a_dlp, a_sp), "tsqbx_eval_pk")
        return outs

    def eval_async(self, density, out, stream=None, p=None, k=None):
        """Enqueue on a CUDA stream (tsqbx_eval_async; tsqbx_eval_async_pk
        when p or k is given or out has an "sp" entry); device tensors only.
        stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        handle = None
        if stream is not None:
            handle = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        a_slp, a_dlp, a_sp = self._out_addrs(out)
        d = self._density_addr(density)
        if p is None and k is None and a_sp is None:
            check(lib().tsqbx_eval_async(self._h, d, a_slp, a_dlp, handle), "tsqbx_eval_async")
        else:
            pp = self.p if p is None else int(p)
            kk = self.k if k is None else float(k)
            check(lib().tsqbx_eval_async_pk(self._h, pp, kk, d, a_slp, a_dlp, a_sp, handle),
                  "tsqbx_eval_async_pk")
        return out

    def submit(self, density, out=None):
        """tsqbx_submit (tsqbx_submit_pk when the plan forms S'): returns
        (ticket, outs); outs are valid once poll() returns True."""
        like = density if _is_torch(density) and density.is_cuda else None
        outs = out if out is not None else self._alloc_out(like)
        a_slp, a_dlp, a_sp = self._out_addrs(outs)
        t = ctypes.c_uint64()
        if a_sp is None:
            check(lib().tsqbx_submit(self._h, self._density_addr(density), a_slp, a_dlp, ctypes.byref(t)),
                  "tsqbx_submit")
        else:
            check(lib().tsqbx_submit_pk(self._h, self.p, self.k, self._density_addr(density), a_slp, a_dlp,
                                        a_sp, ctypes.byref(t)), "tsqbx_submit_pk")
        self._inflight = getattr(self, "_inflight", {})
        self._inflight[t.value] = (outs, getattr(self, "_keep_density", None))
        return t.value, outs


    def submit_multi(self, densities, p=None, k=None, outs=None):
        """tsqbx_submit_multi_layers: every layer of the plan for several
        densities in one evaluation (plans created with max_rhs: the
        Helmholtz single layer, the Laplace single and/or double layer in
        FP64 or df64); returns (ticket, [{layer: out} per density]), valid
        once poll() returns True."""
        n = len(densities)
        helm = self.kernel == "helmholtz"
        cw = np.complex128 if helm else np.float64
        esz = 16 if helm else 8
        layers = [l for l in ("slp", "dlp") if l in self.layers]
        keep = []
        d_addr = (ctypes.c_void_p * n)()
        o_addr = {l: (ctypes.c_void_p * n)() for l in ("slp", "dlp")}
        if outs is None:
            outs = []
            for d in densities:
                if _is_torch(d) and d.is_cuda:
                    import torch
                    tdt = torch.complex128 if helm else torch.float64
                    outs.append({l: torch.empty(self.n_tgt, dtype=tdt, device=d.device) for l in layers})
                else:
                    outs.append({l: np.empty(self.n_tgt, dtype=cw) for l in layers})
        for i, d in enumerate(densities):
            if not _is_torch(d):
                d = np.ascontiguousarray(d, dtype=cw)
            keep.append(d)
            d_addr[i] = _addr(d, self.n_src * esz, "density").value
            for l in layers:
                o_addr[l][i] = _addr(outs[i][l], self.n_tgt * esz, "out_" + l).value
        t = ctypes.c_uint64()
        pp = self.p if p is None else int(p)
        kk = self.k if k is None else float(k)
        check(lib().tsqbx_submit_multi_layers(self._h, pp, kk, n, d_addr,
                                              o_addr["slp"] if "slp" in layers else None,
                                              o_addr["dlp"] if "dlp" in layers else None, ctypes.byref(t)),
              "tsqbx_submit_multi_layers")
        self._inflight = getattr(self, "_inflight", {})
        self._inflight[t.value] = (outs, keep)
        return t.value, outs


class Batch:
    """Many Laplace plans in one persistent launch (tsqbx_batch_*).  The plans
    must outlive the batch."""

    def __init__(self, plans, use_graph=True):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        check(lib().tsqbx_batch_create(arr, len(self.plans), 1 if use_graph else 0, ctypes.byref(h)),
              "tsqbx_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tsqbx_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def eval_async(self, densities, outs, stream=None):
        """densities: list of device tensors; outs: list of {'slp': t, 'dlp': t}."""
        n = len(self.plans)
        ptr = lambda t: None if t is None else t.data_ptr()
        d = (ctypes.c_void_p * n)(*[ptr(x) for x in densities])
        s = (ctypes.c_void_p * n)(*[ptr(o.get("slp")) for o in outs])
        dl = (ctypes.c_void_p * n)(*[ptr(o.get("dlp")) for o in outs])
        handle = None
        if stream is not None:
            handle = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        check(lib().tsqbx_batch_eval_async(self._h, d, s, dl, handle), "tsqbx_batch_eval_async")

    def kernel_ms(self):
        ms = ctypes.c_float()
        check(lib().tsqbx_batch_kernel_ms(self._h, ctypes.byref(ms)), "tsqbx_batch_kernel_ms")
        return float(ms.value)

    def info(self):
        st = _lib.tsqbx_batch_stats()
        check(lib().tsqbx_batch_info(self._h, ctypes.byref(st)), "tsqbx_batch_info")
        return {name: getattr(st, name) for name, _ in st._fields_}


class Server:
    """Request-serving runtime (tsqbx_server_*): register geometries, submit
    evaluations as they arrive, poll for completion, read p50/p99 latency."""

    def __init__(self, device=0, hbm_budget=16 << 30, max_inflight=64, size_priority=False,
                 laplace_fp64_path="fp64"):
        """size_priority: build plans whose streams are prioritised by size
        (tsqbx_server_set_size_priority): short evaluations overtake long ones.
        laplace_fp64_path: "fp64" or "df64", the kernels that serve Laplace
        requests asking for FP64 (tsqbx_server_set_laplace_fp64_path)."""
        h = ctypes.c_void_p()
        check(lib().tsqbx_server_create(int(device), int(hbm_budget), int(max_inflight), ctypes.byref(h)),
              "tsqbx_server_create")
        self._h = h
        self._geoms = {}
        self._pending = {}
        if size_priority:
            check(lib().tsqbx_server_set_size_priority(self._h, 1), "tsqbx_server_set_size_priority")
        if laplace_fp64_path != "fp64":
            check(lib().tsqbx_server_set_laplace_fp64_path(self._h, _PRECISIONS[laplace_fp64_path]),
                  "tsqbx_server_set_laplace_fp64_path")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tsqbx_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_geometry(self, g, with_normals=True):
        geo, keep = marshal_geometry(g, with_normals,
                                     with_tgt_normals=with_normals and getattr(g, "tgt_normal", None) is not None)
        gid = ctypes.c_int()
        check(lib().tsqbx_server_add_geometry(self._h, ctypes.byref(geo), ctypes.byref(gid)),
              "tsqbx_server_add_geometry")
        self._geoms[gid.value] = (int(geo.n_src), int(geo.n_tgt))
        return gid.value

    def prepare(self, gid, kernel="laplace", layers=("slp",), p=5, k=0.0, precision="fp64"):
        opt = make_options(kernel, layers, p, k, precision)
        check(lib().tsqbx_server_prepare(self._h, int(gid), ctypes.byref(opt)), "tsqbx_server_prepare")

    def submit(self, gid, density, kernel="laplace", layers=("slp",), p=5, k=0.0, precision="fp64"):
        """Queue a request; returns (request_id, outs) with host output arrays
        that are valid once poll() returns True."""
        if gid not in self._geoms:
            raise TsqbxError(_lib.TSQBX_E_INVAL, "tsqbx_server_submit")
        n_src, n_tgt = self._geoms[gid]
        cplx = kernel == "helmholtz"
        dens = np.ascontiguousarray(density, dtype=np.complex128 if cplx else np.float64)
        outs = {l: np.empty(n_tgt, dtype=np.complex128 if cplx else np.float64) for l in layers}
        opt = make_options(kernel, layers, p, k, precision)
        rid = ctypes.c_uint64()
        check(lib().tsqbx_server_submit(self._h, int(gid), ctypes.byref(opt), ctypes.c_void_p(dens.ctypes.data),
                                        None if "slp" not in outs else ctypes.c_void_p(outs["slp"].ctypes.data),
                                        None if "dlp" not in outs else ctypes.c_void_p(outs["dlp"].ctypes.data),
                                        None if "sp" not in outs else ctypes.c_void_p(outs["sp"].ctypes.data),
                                        ctypes.byref(rid)), "tsqbx_server_submit")
        self._pending[rid.value] = outs
        return rid.value, outs

    def poll(self, rid, timeout_us=0):
        """True once done (raises TsqbxError if the request failed), False while pending."""
        rc = lib().tsqbx_server_poll(self._h, ctypes.c_uint64(rid), int(timeout_us))
        if rc == _lib.TSQBX_PENDING:
            return False
        if rc == _lib.TSQBX_E_TIMEOUT:
            return False
        self._pending.pop(rid, None)
        check(rc, "tsqbx_server_poll")
        return True

    def stats(self):
        st = _lib.tsqbx_server_stats()
        check(lib().tsqbx_server_get_stats(self._h, ctypes.byref(st)), "tsqbx_server_get_stats")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def reset_stats(self):
        check(lib().tsqbx_server_reset_stats(self._h), "tsqbx_server_reset_stats")


class Octree:
    """The GIGAQBX octree and near-field lists built on the GPU
    (tsqbx_octree_build).  Attributes mirror the host builder's: per box
    level, center (3, n_boxes), halfwidth, parent, src_begin, src_end,
    n_owned_ctr, is_leaf; src_perm, ctr_box; near_start, near_begin,
    near_end; stats."""

    def __init__(self, src_xyz, ctr_xyz, ctr_radius, n_max=64, t_f=0.9, n_mpole=40, device=0):
        s = np.ascontiguousarray(np.asarray(src_xyz, dtype=np.float64).T)      # (3, n) from (n, 3)
        c = np.ascontiguousarray(np.asarray(ctr_xyz, dtype=np.float64).T)
        r = np.ascontiguousarray(ctr_radius, dtype=np.float64)
        self.n_src, self.n_ctr = s.shape[1], c.shape[1]
        h = ctypes.c_void_p()
        check(lib().tsqbx_octree_build(self.n_src, _ptr(s, ctypes.c_double), self.n_ctr,
                                       _ptr(c, ctypes.c_double), _ptr(r, ctypes.c_double), int(n_max),
                                       float(t_f), int(n_mpole), int(device), ctypes.byref(h)),
              "tsqbx_octree_build")
        try:
            st = _lib.tsqbx_octree_stats()
            check(lib().tsqbx_octree_info(h, ctypes.byref(st)), "tsqbx_octree_info")
            self.stats = {name: getattr(st, name) for name, _ in st._fields_}
            nb = int(st.n_boxes)
            self.n_boxes = nb
            i32 = lambda n: np.zeros(max(n, 1), np.int32)
            self.level, self.parent, self.src_begin, self.src_end = i32(nb), i32(nb), i32(nb), i32(nb)
            self.n_owned_ctr, self.is_leaf = i32(nb), i32(nb)
            self.center, self.halfwidth = np.zeros(3 * max(nb, 1)), np.zeros(max(nb, 1))
            check(lib().tsqbx_octree_boxes(h, _ptr(self.level, ctypes.c_int32), _ptr(self.center, ctypes.c_double),
                                           _ptr(self.halfwidth, ctypes.c_double), _ptr(self.parent, ctypes.c_int32),
                                           _ptr(self.src_begin, ctypes.c_int32), _ptr(self.src_end, ctypes.c_int32),
                                           _ptr(self.n_owned_ctr, ctypes.c_int32),
                                           _ptr(self.is_leaf, ctypes.c_int32)), "tsqbx_octree_boxes")
            for name in ("level", "parent", "src_begin", "src_end", "n_owned_ctr", "is_leaf", "halfwidth"):
                setattr(self, name, getattr(self, name)[:nb])
            self.center = self.center[:3 * nb].reshape(3, nb)
            self.src_perm, self.ctr_box = i32(self.n_src), i32(self.n_ctr)
            check(lib().tsqbx_octree_order(h, _ptr(self.src_perm, ctypes.c_int32), _ptr(self.ctr_box, ctypes.c_int32)),
                  "tsqbx_octree_order")
            self.src_perm, self.ctr_box = self.src_perm[:self.n_src], self.ctr_box[:self.n_ctr]
            nnz = int(st.near_nnz)
            self.near_start = np.zeros(nb + 1, np.int64)
            self.near_begin, self.near_end = i32(nnz), i32(nnz)
            check(lib().tsqbx_octree_near(h, _ptr(self.near_start, ctypes.c_int64),
                                          _ptr(self.near_begin, ctypes.c_int32), _ptr(self.near_end, ctypes.c_int32)),
                  "tsqbx_octree_near")
            self.near_begin, self.near_end = self.near_begin[:nnz], self.near_end[:nnz]
        finally:
            lib().tsqbx_octree_destroy(h)


def octree_lists(src_xyz, ctr_xyz, ctr_radius, n_max=64, t_f=0.9, n_mpole=40, device=0):
    """GPU-built octree and near-field lists, packaged as pair lists: returns
    (tree, src_perm, ctr_order, ctr_group, group_range_start, range_begin,
    range_end).  Sources must be permuted by src_perm and centers by
    ctr_order (grouped by owning box); the ranges index the permuted sources."""
    tree = Octree(src_xyz, ctr_xyz, ctr_radius, n_max, t_f, n_mpole, device)
    target_boxes = np.nonzero(tree.n_owned_ctr > 0)[0]
    gid = -np.ones(tree.n_boxes, np.int64)
    gid[target_boxes] = np.arange(len(target_boxes))
    ctr_g = gid[tree.ctr_box]
    ctr_order = np.argsort(ctr_g, kind="stable")
    ctr_group = ctr_g[ctr_order].astype(np.int32)
    counts = tree.near_start[target_boxes + 1] - tree.near_start[target_boxes]
    grs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    sel = (np.concatenate([np.arange(tree.near_start[b], tree.near_start[b + 1]) for b in target_boxes])
           if len(target_boxes) else np.zeros(0, np.int64))
    rb = tree.near_begin[sel].astype(np.int32)
    re = tree.near_end[sel].astype(np.int32)
    return tree, tree.src_perm.astype(np.int64), ctr_order, ctr_group, grs, rb, re


def poll(ticket, timeout_us=0):
    """tsqbx_poll: True when done, False while pending (timeout_us == 0)."""
    rc = lib().tsqbx_poll(ctypes.c_uint64(ticket), int(timeout_us))
    if rc == _lib.TSQBX_PENDING:
        return False
    check(rc, "tsqbx_poll")
    return True


def measure_pipe_peaks(device=0):
    """tsqbx_measure_pipe_peaks: measured FP64 / FP32 / packed-FP32 FMA
    throughput (TFLOP/s, FMA = 2 flops) and the device's SM count."""
    r = _lib.tsqbx_pipe_peaks()
    check(lib().tsqbx_measure_pipe_peaks(int(device), ctypes.byref(r)), "tsqbx_measure_pipe_peaks")
    return {"fp64_tflops": r.fp64_tflops, "fp32_tflops": r.fp32_tflops, "fp32x2_tflops": r.fp32x2_tflops,
            "sm_count": r.sm_count, "ms": {"fp64": r.ms_fp64, "fp32": r.ms_fp32, "fp32x2": r.ms_fp32x2}}
