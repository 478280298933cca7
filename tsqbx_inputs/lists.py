"""Grouped CSR pair lists: radius lists and GIGAQBX octree lists.

Output layout (the library's): centers are partitioned into groups; a group
owns a CSR of half-open source index ranges [range_begin, range_end), and every
target of every center in the group is paired with every listed source.
"""
import ctypes

import numpy as np

from . import build as _build


def lists_to_csr(lists):
    """Sorted per-group index arrays -> (group_range_start, range_begin, range_end),
    merging runs of consecutive indices into ranges."""
    lens = np.array([len(x) for x in lists], dtype=np.int64)
    n = len(lists)
    if lens.sum() == 0:
        return np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32)
    flat = np.concatenate([np.asarray(x, dtype=np.int64) for x in lists])
    owner = np.repeat(np.arange(n), lens)
    brk = np.ones(len(flat), dtype=bool)
    brk[1:] = (owner[1:] != owner[:-1]) | (flat[1:] != flat[:-1] + 1)
    starts = np.nonzero(brk)[0]
    ends = np.append(starts[1:], len(flat))
    rb = flat[starts].astype(np.int32)
    re = (flat[ends - 1] + 1).astype(np.int32)
    counts = np.bincount(owner[starts], minlength=n)
    grs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return grs, rb, re


def radius_lists(src_xyz, ctr_xyz, radii):
    """Per center: all sources with |s - c| <= radius (one group per center)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(src_xyz)
    res = tree.query_ball_point(ctr_xyz, r=radii)
    return lists_to_csr([np.sort(np.asarray(x, dtype=np.int64)) for x in res])


def nearest_lists(src_xyz, ctr_xyz, counts):
    """Per center: its counts[c] nearest sources (one group per center)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(src_xyz)
    kmax = int(min(max(counts.max(), 1), len(src_xyz)))
    _, idx = tree.query(ctr_xyz, k=kmax)
    idx = idx.reshape(len(ctr_xyz), -1)
    return lists_to_csr([np.sort(idx[c, :min(int(counts[c]), kmax)]) for c in range(len(ctr_xyz))])


# ------------------------------------------------------------------ octree

LIST_KINDS = {"L1": 0, "L3close": 1, "L3far": 2, "L4close": 3, "L2": 4, "L4far": 5,
              "L3": 6, "L4": 7}

_libs = {}


def _octlib(path=None):
    """The builder library, compiled on first use; `path` loads another build of
    the same source (the tests load copies with planted mistakes)."""
    key = path or ""
    if key not in _libs:
        L = ctypes.CDLL(path or _build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        i32 = ctypes.POINTER(ctypes.c_int32)
        i64 = ctypes.POINTER(ctypes.c_int64)
        L.oct_build.restype = ctypes.c_void_p
        L.oct_build.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, dp, dp, ctypes.c_int,
                                ctypes.c_double, ctypes.c_int]
        L.oct_free.argtypes = [ctypes.c_void_p]
        L.oct_n_boxes.restype = ctypes.c_int64
        L.oct_n_boxes.argtypes = [ctypes.c_void_p]
        L.oct_box_info.argtypes = [ctypes.c_void_p, i32, dp, dp, i32, i32, i32, i32, i32]
        L.oct_src_perm.argtypes = [ctypes.c_void_p, i32]
        L.oct_ctr_box.argtypes = [ctypes.c_void_p, i32]
        L.oct_list_nnz.restype = ctypes.c_int64
        L.oct_list_nnz.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oct_list.restype = ctypes.c_int
        L.oct_list.argtypes = [ctypes.c_void_p, ctypes.c_int, i64, i32]
        L.oct_near_nnz.restype = ctypes.c_int64
        L.oct_near_nnz.argtypes = [ctypes.c_void_p]
        L.oct_near_ranges.argtypes = [ctypes.c_void_p, i64, i32, i32]
        _libs[key] = L
    return _libs[key]


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class Octree:
    """GIGAQBX octree (Sec. 3.1) over sources and QBX centers, with the
    interaction lists of Sec. 3.2.  Sources are reordered depth first, so every
    box's sources form one contiguous range; `src_perm[i]` is the original
    index of sorted source i."""

    def __init__(self, src_xyz, ctr_xyz, ctr_radius, n_max=64, t_f=0.9, n_mpole=40, lib_path=None):
        L = _octlib(lib_path)
        self.t_f, self.n_mpole = float(t_f), int(n_mpole)
        s = np.ascontiguousarray(np.asarray(src_xyz, dtype=np.float64).T)
        c = np.ascontiguousarray(np.asarray(ctr_xyz, dtype=np.float64).T)
        r = np.ascontiguousarray(ctr_radius, dtype=np.float64)
        self.n_src, self.n_ctr = s.shape[1], c.shape[1]
        h = L.oct_build(self.n_src, _ptr(s, ctypes.c_double), self.n_ctr, _ptr(c, ctypes.c_double),
                        _ptr(r, ctypes.c_double), int(n_max), float(t_f), int(n_mpole))
        if not h:
            raise ValueError("octree build rejected its input")
        try:
            nb = int(L.oct_n_boxes(h))
            self.n_boxes = nb
            self.level = np.zeros(nb, np.int32)
            self.center = np.zeros(3 * nb)
            self.halfwidth = np.zeros(nb)
            self.parent = np.zeros(nb, np.int32)
            self.src_begin = np.zeros(nb, np.int32)
            self.src_end = np.zeros(nb, np.int32)
            self.n_owned_ctr = np.zeros(nb, np.int32)
            self.is_leaf = np.zeros(nb, np.int32)
            L.oct_box_info(h, _ptr(self.level, ctypes.c_int32), _ptr(self.center, ctypes.c_double),
                           _ptr(self.halfwidth, ctypes.c_double), _ptr(self.parent, ctypes.c_int32),
                           _ptr(self.src_begin, ctypes.c_int32), _ptr(self.src_end, ctypes.c_int32),
                           _ptr(self.n_owned_ctr, ctypes.c_int32), _ptr(self.is_leaf, ctypes.c_int32))
            self.center = self.center.reshape(3, nb)
            self.src_perm = np.zeros(self.n_src, np.int32)
            L.oct_src_perm(h, _ptr(self.src_perm, ctypes.c_int32))
            self.ctr_box = np.zeros(self.n_ctr, np.int32)
            L.oct_ctr_box(h, _ptr(self.ctr_box, ctypes.c_int32))
            self.lists = {}
            for name, kind in LIST_KINDS.items():
                nnz = int(L.oct_list_nnz(h, kind))
                st = np.zeros(nb + 1, np.int64)
                bx = np.zeros(max(nnz, 1), np.int32)
                L.oct_list(h, kind, _ptr(st, ctypes.c_int64), _ptr(bx, ctypes.c_int32))
                self.lists[name] = (st, bx[:nnz])
            nnz = int(L.oct_near_nnz(h))
            self.near_start = np.zeros(nb + 1, np.int64)
            self.near_begin = np.zeros(max(nnz, 1), np.int32)
            self.near_end = np.zeros(max(nnz, 1), np.int32)
            L.oct_near_ranges(h, _ptr(self.near_start, ctypes.c_int64),
                              _ptr(self.near_begin, ctypes.c_int32), _ptr(self.near_end, ctypes.c_int32))
            self.near_begin = self.near_begin[:nnz]
            self.near_end = self.near_end[:nnz]
        finally:
            L.oct_free(h)

    def box_list(self, name, b):
        st, bx = self.lists[name]
        return bx[st[b]:st[b + 1]]

    def ancestors(self, b):
        out = []
        while b >= 0:
            out.append(b)
            b = int(self.parent[b])
        return out


def octree_lists(src_xyz, ctr_xyz, ctr_radius, n_max=64, t_f=0.9, n_mpole=40):
    """Build the octree and the near-field lists List 1 + List 3 close + List 4
    close (the sources of L^{qbx,near}_c, Alg. 1 Stages 3, 5(a), 6(a)).

    Returns (tree, src_perm, ctr_order, ctr_group, group_range_start,
    range_begin, range_end): sources must be permuted by src_perm and centers
    by ctr_order (grouped by owning box); ranges index the permuted sources."""
    tree = Octree(src_xyz, ctr_xyz, ctr_radius, n_max, t_f, n_mpole)
    target_boxes = np.nonzero(tree.n_owned_ctr > 0)[0]
    gid = -np.ones(tree.n_boxes, np.int64)
    gid[target_boxes] = np.arange(len(target_boxes))
    ctr_g = gid[tree.ctr_box]
    ctr_order = np.argsort(ctr_g, kind="stable")
    ctr_group = ctr_g[ctr_order].astype(np.int32)
    counts = tree.near_start[target_boxes + 1] - tree.near_start[target_boxes]
    grs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    sel = np.concatenate([np.arange(tree.near_start[b], tree.near_start[b + 1])
                          for b in target_boxes]) if len(target_boxes) else np.zeros(0, np.int64)
    rb = tree.near_begin[sel].astype(np.int32)
    re = tree.near_end[sel].astype(np.int32)
    return tree, tree.src_perm.astype(np.int64), ctr_order, ctr_group, grs, rb, re
