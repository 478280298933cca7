"""FP64 CPU oracle for the TSQBX near-field step (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may use this package; the product
(the ``libtsqbx`` C ABI and its Python binding) never imports it and shares no
code with it.

Every function takes a *geometry* object: anything with the numpy attributes
``src_xyz (3, n_src) f64``, ``src_weight (n_src,)``, ``src_normal (3, n_src)``
or None, ``ctr_xyz (3, n_ctr)``, ``tgt_xyz (3, n_tgt)``, ``tgt_center
(n_tgt,) i32``, ``tgt_normal (3, n_tgt)`` or None, ``ctr_group (n_ctr,) i32``,
``group_range_start (n_group+1,) i64``, ``range_begin``/``range_end (nnz,) i32``.

Paths (see oracle.c for the formulas and their paper citations):
  * ``tsqbx_laplace`` / ``tsqbx_helmholtz`` -- path A, Appendix A written out;
  * ``qbx_laplace`` / ``qbx_helmholtz`` -- path B, conventional local
    coefficients (Sec. 2.1 eqs. local-coeffs, local-expansion);
  * ``point_potential`` -- the un-expanded kernels over the same lists.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
P_MAX = 40

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class _Geom(ctypes.Structure):
    _fields_ = [
        ("n_src", _i64), ("src_xyz", _dp), ("src_weight", _dp), ("src_normal", _dp),
        ("n_ctr", _i64), ("ctr_xyz", _dp),
        ("n_tgt", _i64), ("tgt_xyz", _dp), ("tgt_center", _i32p), ("tgt_normal", _dp),
        ("n_group", _i64), ("ctr_group", _i32p), ("group_range_start", _i64p),
        ("range_begin", _i32p), ("range_end", _i32p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB lets the mutation tests load a deliberately broken copy
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        gp = ctypes.POINTER(_Geom)
        for name in ("oracle_tsqbx_laplace", "oracle_qbx_laplace"):
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = [gp, ctypes.c_int, _dp, _i64p, _i64, _dp, _dp, _dp]
        for name in ("oracle_tsqbx_helmholtz", "oracle_qbx_helmholtz"):
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = [gp, ctypes.c_int, ctypes.c_double, _dp, _i64p, _i64, _dp, _dp, _dp]
        L.oracle_point_potential.restype = ctypes.c_int
        L.oracle_point_potential.argtypes = [gp, ctypes.c_int, ctypes.c_double, _dp, _i64p, _i64,
                                             _dp, _dp, _dp]
        L.oracle_count_pairs.restype = ctypes.c_int64
        L.oracle_count_pairs.argtypes = [gp]
        L.oracle_count_divergent.restype = ctypes.c_int
        L.oracle_count_divergent.argtypes = [gp, _i64p, _i64p]
        L.oracle_legendre.restype = ctypes.c_int
        L.oracle_legendre.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        for name in ("oracle_sph_jn", "oracle_sph_yn", "oracle_sph_jn_deriv", "oracle_sph_yn_deriv"):
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        L.oracle_sph_harm.restype = ctypes.c_int
        L.oracle_sph_harm.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _dp, _dp]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        L.oracle_set_num_threads.restype = None
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class _Bound:
    """Keeps contiguous copies alive while the C struct points at them."""

    def __init__(self, g):
        def f64(a):
            return None if a is None else np.ascontiguousarray(a, dtype=np.float64)

        def i32(a):
            return np.ascontiguousarray(a, dtype=np.int32)

        self.src_xyz = f64(g.src_xyz)
        self.src_weight = f64(g.src_weight)
        self.src_normal = f64(getattr(g, "src_normal", None))
        self.ctr_xyz = f64(g.ctr_xyz)
        self.tgt_xyz = f64(g.tgt_xyz)
        self.tgt_center = i32(g.tgt_center)
        self.tgt_normal = f64(getattr(g, "tgt_normal", None))
        self.ctr_group = i32(g.ctr_group)
        self.group_range_start = np.ascontiguousarray(g.group_range_start, dtype=np.int64)
        self.range_begin = i32(g.range_begin)
        self.range_end = i32(g.range_end)
        self.n_src = self.src_weight.shape[0]
        self.n_ctr = self.ctr_xyz.shape[1]
        self.n_tgt = self.tgt_xyz.shape[1]
        self.n_group = self.group_range_start.shape[0] - 1
        self.s = _Geom(
            self.n_src, _p(self.src_xyz, ctypes.c_double), _p(self.src_weight, ctypes.c_double),
            _p(self.src_normal, ctypes.c_double),
            self.n_ctr, _p(self.ctr_xyz, ctypes.c_double),
            self.n_tgt, _p(self.tgt_xyz, ctypes.c_double), _p(self.tgt_center, ctypes.c_int32),
            _p(self.tgt_normal, ctypes.c_double),
            self.n_group, _p(self.ctr_group, ctypes.c_int32),
            _p(self.group_range_start, ctypes.c_int64),
            _p(self.range_begin, ctypes.c_int32), _p(self.range_end, ctypes.c_int32))


def _subset(subset, n_tgt):
    if subset is None:
        return None, n_tgt
    s = np.ascontiguousarray(subset, dtype=np.int64)
    return s, s.shape[0]


def _run(fn, g, head_args, density, subset, slp, dlp, sp, complex_out):
    b = _Bound(g)
    sub, n = _subset(subset, b.n_tgt)
    width = 2 if complex_out else 1
    outs = [np.zeros(n * width) if flag else None for flag in (slp, dlp, sp)]
    dens = np.ascontiguousarray(density, dtype=np.complex128 if complex_out else np.float64)
    dens_f = dens.view(np.float64) if complex_out else dens
    rc = fn(ctypes.byref(b.s), *head_args, _p(dens_f, ctypes.c_double),
            _p(sub, ctypes.c_int64), n, *[_p(o, ctypes.c_double) for o in outs])
    if rc != 0:
        raise ValueError(f"oracle rejected the input (status {rc})")
    res = {}
    for name, o in zip(("slp", "dlp", "sp"), outs):
        if o is not None:
            res[name] = o.view(np.complex128) if complex_out else o
    return res


def tsqbx_laplace(g, p, density, subset=None, slp=True, dlp=False, sp=False):
    """Path A, Laplace (Appendix A).  Returns {'slp','dlp','sp'} arrays (1/(4 pi) included)."""
    return _run(lib().oracle_tsqbx_laplace, g, (int(p),), density, subset, slp, dlp, sp, False)


def tsqbx_helmholtz(g, p, k, density, subset=None, slp=True, dlp=False, sp=False):
    """Path A, Helmholtz (Appendix A), complex density and outputs."""
    return _run(lib().oracle_tsqbx_helmholtz, g, (int(p), float(k)), density, subset,
                slp, dlp, sp, True)


def qbx_laplace(g, p, density, subset=None, slp=True, dlp=False, sp=False):
    """Path B, conventional spherical-harmonic QBX (Sec. 2.1)."""
    return _run(lib().oracle_qbx_laplace, g, (int(p),), density, subset, slp, dlp, sp, False)


def qbx_helmholtz(g, p, k, density, subset=None, slp=True, dlp=False, sp=False):
    """Path B for Helmholtz (addition theorem of Appendix A with eq. legendre-addition-identity)."""
    return _run(lib().oracle_qbx_helmholtz, g, (int(p), float(k)), density, subset,
                slp, dlp, sp, True)


def point_potential(g, kernel, density, k=0.0, subset=None, slp=True, dlp=False, sp=False):
    """Un-expanded kernels over the same lists; kernel 'laplace' or 'helmholtz'."""
    kid = {"laplace": 0, "helmholtz": 1}[kernel]
    return _run(lib().oracle_point_potential, g, (kid, float(k)), density, subset,
                slp, dlp, sp, kid == 1)


def count_pairs(g):
    b = _Bound(g)
    n = lib().oracle_count_pairs(ctypes.byref(b.s))
    if n < 0:
        raise ValueError("invalid geometry")
    return int(n)


def count_divergent(g):
    """(pairs with |t-c| >= |s-c|, pairs with s == c)."""
    b = _Bound(g)
    nd, nz = ctypes.c_int64(), ctypes.c_int64()
    if lib().oracle_count_divergent(ctypes.byref(b.s), ctypes.byref(nd), ctypes.byref(nz)):
        raise ValueError("invalid geometry")
    return int(nd.value), int(nz.value)


def legendre(p, x):
    P, dP = np.zeros(p + 1), np.zeros(p + 1)
    if lib().oracle_legendre(int(p), float(x), _p(P, ctypes.c_double), _p(dP, ctypes.c_double)):
        raise ValueError("bad order")
    return P, dP


def _bessel(name, nmax, z):
    out = np.zeros(nmax + 1)
    if getattr(lib(), name)(int(nmax), float(z), _p(out, ctypes.c_double)):
        raise ValueError("bad argument")
    return out


def sph_jn(nmax, z):
    return _bessel("oracle_sph_jn", nmax, z)


def sph_yn(nmax, z):
    return _bessel("oracle_sph_yn", nmax, z)


def sph_jn_deriv(nmax, z):
    return _bessel("oracle_sph_jn_deriv", nmax, z)


def sph_yn_deriv(nmax, z):
    return _bessel("oracle_sph_yn_deriv", nmax, z)


def sph_harm(p, v):
    """Y_n^m (eq. sph-harm, no Condon-Shortley phase) at direction v; index n*n+n+m."""
    re, im = np.zeros((p + 1) ** 2), np.zeros((p + 1) ** 2)
    if lib().oracle_sph_harm(int(p), float(v[0]), float(v[1]), float(v[2]),
                             _p(re, ctypes.c_double), _p(im, ctypes.c_double)):
        raise ValueError("bad argument")
    return re + 1j * im


def num_threads():
    return int(lib().oracle_num_threads())


def set_num_threads(n):
    lib().oracle_set_num_threads(int(n))
