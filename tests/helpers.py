"""Small hand-built geometries for the oracle pins and parity tests, and the
builder of the test-only native shims."""
import os

import numpy as np

from tsqbx_inputs.geometry import Geometry
from tsqbx_inputs.lists import lists_to_csr


def random_unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def cloud_geometry(rng, n_ctr=4, n_src=40, q_max=0.7, tgt_per_ctr=1, list_frac=1.0,
                   dup=False, rho_zero=False):
    """Centers in a box, sources scattered around them, targets inside each
    center's ball with |t-c| <= q_max * min |s-c| over its list (convergent).
    Every center is its own group listing a random subset of the sources."""
    ctr = rng.uniform(-1, 1, (n_ctr, 3))
    src = rng.uniform(-2, 2, (n_src, 3))
    w = rng.uniform(0.5, 1.5, n_src)
    nrm = random_unit(rng, n_src)
    lists = []
    for c in range(n_ctr):
        k = max(1, int(round(list_frac * n_src)))
        sel = np.sort(rng.choice(n_src, size=k, replace=False))
        if dup:
            sel = np.sort(np.concatenate([sel, sel[: max(1, k // 4)]]))
        lists.append(sel)
    grs, rb, re = lists_to_csr([np.unique(x) for x in lists])
    if dup:   # append a duplicated range per center (summed twice)
        nrb, nre, ngrs = [], [], [0]
        for c in range(n_ctr):
            a, b = grs[c], grs[c + 1]
            nrb += list(rb[a:b]) + [rb[a]]
            nre += list(re[a:b]) + [re[a]]
            ngrs.append(len(nrb))
        rb, re, grs = np.array(nrb, np.int32), np.array(nre, np.int32), np.array(ngrs, np.int64)
    tgt, tc, tn = [], [], []
    for c in range(n_ctr):
        members = np.concatenate([np.arange(rb[i], re[i]) for i in range(grs[c], grs[c + 1])])
        Rmin = np.linalg.norm(src[members] - ctr[c], axis=1).min()
        for j in range(tgt_per_ctr):
            if rho_zero and j == 0:
                tgt.append(ctr[c].copy())
            else:
                d = random_unit(rng, 1)[0]
                tgt.append(ctr[c] + rng.uniform(0.05, q_max) * Rmin * d)
            tc.append(c)
            tn.append(random_unit(rng, 1)[0])
    tgt = np.array(tgt)
    return Geometry(np.ascontiguousarray(src.T), w, np.ascontiguousarray(nrm.T),
                    np.ascontiguousarray(ctr.T), np.full(n_ctr, 0.1),
                    np.ascontiguousarray(tgt.T), np.array(tc, np.int32),
                    np.ascontiguousarray(np.array(tn).T), np.arange(n_ctr, dtype=np.int32),
                    grs, rb, re)


def single_pair(t, c, s, n_s=None, n_t=None, w=1.0):
    """One target, one center, one source."""
    n_s = np.array([0.0, 0.0, 1.0]) if n_s is None else np.asarray(n_s, float)
    n_t = np.array([0.0, 0.0, 1.0]) if n_t is None else np.asarray(n_t, float)
    col = lambda v: np.asarray(v, float).reshape(3, 1)
    return Geometry(col(s), np.array([w]), col(n_s), col(c), np.array([0.1]), col(t),
                    np.array([0], np.int32), col(n_t), np.array([0], np.int32),
                    np.array([0, 1], np.int64), np.array([0], np.int32), np.array([1], np.int32))


def native_shim(name, deps=()):
    """Build tests/native/<name>.cu (a test-only C shim around library headers)
    into tests/native/_build/lib<name>.so when it is older than its sources;
    return the path, or None without nvcc."""
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        return None
    src = os.path.join(root, "tests", "native", name + ".cu")
    out = os.path.join(root, "tests", "native", "_build", "lib" + name + ".so")
    csrc = os.path.join(root, "paper_1811_01110_gb300", "csrc")
    allsrc = [src, os.path.join(root, "include", "tsqbx.h")] + [os.path.join(csrc, f) for f in os.listdir(csrc)]
    if not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(d) for d in allsrc):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "-shared",
                        "-I", os.path.join(root, "include"), src, "-o", out + ".tmp"],
                       check=True, capture_output=True)
        os.replace(out + ".tmp", out)
    return out
