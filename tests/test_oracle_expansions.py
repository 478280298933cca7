"""Pins for the oracle's expansions (path A, Appendix A; path B, Sec. 2.1).

Each test ties the oracle to something other than itself: the addition
theorem (A == B, eq. tsqbx), the point kernel the series converges to
(eq. laplace-potential-expansion, DLMF 10.60) with the closed-form tail
bound, closed forms for special geometries, finite differences for the
normal derivatives, and a 50-digit brute force of tiny cases.
"""
import numpy as np
import pytest

import oracle
from helpers import cloud_geometry, single_pair

mpmath = pytest.importorskip("mpmath")

FOURPI = 4 * np.pi


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ----------------------------------------------------- path A == path B

@pytest.mark.parametrize("p", [0, 1, 3, 6, 10])
def test_laplace_paths_agree(rng, p):
    g = cloud_geometry(rng, n_ctr=5, n_src=30, tgt_per_ctr=2)
    mu = rng.standard_normal(g.n_src)
    a = oracle.tsqbx_laplace(g, p, mu, slp=True, dlp=True, sp=True)
    b = oracle.qbx_laplace(g, p, mu, slp=True, dlp=True, sp=True)
    for k in ("slp", "dlp", "sp"):
        assert rel(a[k], b[k]) < 1e-12, k


@pytest.mark.parametrize("p,k", [(0, 1.0), (3, 5.0), (8, 10.0), (12, 10.0), (12, 0.5)])
def test_helmholtz_paths_agree(rng, p, k):
    g = cloud_geometry(rng, n_ctr=4, n_src=25, tgt_per_ctr=2)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    a = oracle.tsqbx_helmholtz(g, p, k, mu, slp=True, dlp=True, sp=True)
    b = oracle.qbx_helmholtz(g, p, k, mu, slp=True, dlp=True, sp=True)
    for key in ("slp", "dlp", "sp"):
        assert rel(a[key], b[key]) < 1e-11, key


def test_target_at_center_paths_agree(rng):
    g = cloud_geometry(rng, n_ctr=3, n_src=20, tgt_per_ctr=2, rho_zero=True)
    mu = rng.standard_normal(g.n_src)
    a = oracle.tsqbx_laplace(g, 7, mu, slp=True, dlp=True)
    b = oracle.qbx_laplace(g, 7, mu, slp=True, dlp=True)
    assert rel(a["slp"], b["slp"]) < 1e-12 and rel(a["dlp"], b["dlp"]) < 1e-12
    mz = mu + 0.5j
    a = oracle.tsqbx_helmholtz(g, 7, 3.0, mz, slp=True, dlp=True)
    b = oracle.qbx_helmholtz(g, 7, 3.0, mz, slp=True, dlp=True)
    assert rel(a["slp"], b["slp"]) < 1e-12 and rel(a["dlp"], b["dlp"]) < 1e-12
    # S' at t = c: both paths take the limit along n_t
    a = oracle.tsqbx_laplace(g, 7, mu, sp=True)["sp"]
    b = oracle.qbx_laplace(g, 7, mu, sp=True)["sp"]
    assert rel(a, b) < 1e-12
    a = oracle.tsqbx_helmholtz(g, 7, 3.0, mz, sp=True)["sp"]
    b = oracle.qbx_helmholtz(g, 7, 3.0, mz, sp=True)["sp"]
    assert rel(a, b) < 1e-12


# ------------------------------------------------------ special geometries

def test_p0_and_rho0_reduce_to_monopole(rng):
    g = cloud_geometry(rng, n_ctr=3, n_src=15, tgt_per_ctr=2, rho_zero=True)
    mu = rng.standard_normal(g.n_src)
    # p = 0: G^(0) = 1/(4 pi R) for every target
    u0 = oracle.tsqbx_laplace(g, 0, mu)["slp"]
    S, C, T = g.src_xyz.T, g.ctr_xyz.T, g.tgt_xyz.T
    for i in range(g.n_tgt):
        c = g.tgt_center[i]
        idx = np.concatenate([np.arange(g.range_begin[r], g.range_end[r])
                              for r in range(g.group_range_start[c], g.group_range_start[c + 1])])
        R = np.linalg.norm(S[idx] - C[c], axis=1)
        assert u0[i] == pytest.approx(np.sum(g.src_weight[idx] * mu[idx] / (FOURPI * R)), rel=1e-13)
        if np.allclose(T[i], C[c]):
            # rho = 0: every order gives the monopole; DLP = -n.(s-c)/(4 pi R^3);
            # S' = n_t.(s-c)/(4 pi R^3)
            u = oracle.tsqbx_laplace(g, 9, mu, subset=[i], slp=True, dlp=True, sp=True)
            wm = g.src_weight[idx] * mu[idx]
            sc = S[idx] - C[c]
            ns = g.src_normal.T[idx]
            nt = g.tgt_normal.T[i]
            assert u["slp"][0] == pytest.approx(np.sum(wm / (FOURPI * R)), rel=1e-13)
            assert u["dlp"][0] == pytest.approx(
                np.sum(-wm * np.einsum("ij,ij->i", ns, sc) / (FOURPI * R ** 3)), rel=1e-12)
            assert u["sp"][0] == pytest.approx(np.sum(wm * (sc @ nt) / (FOURPI * R ** 3)), rel=1e-12)


@pytest.mark.parametrize("sgn", [1.0, -1.0])
@pytest.mark.parametrize("p", [1, 4, 9, 20])
def test_collinear_geometric_series(sgn, p):
    """t-c parallel (sgn=1) or antiparallel (sgn=-1) to s-c: P_n(+-1) = (+-1)^n,
    so G^(p) = (1/4 pi R) sum_n (sgn q)^n = (1 - (sgn q)^{p+1}) / (1 - sgn q) / (4 pi R)."""
    c = np.array([0.1, -0.2, 0.3])
    d = np.array([1.0, 2.0, -2.0]) / 3.0
    R, q = 0.8, 0.45
    g = single_pair(c + sgn * q * R * d, c, c + R * d)
    u = oracle.tsqbx_laplace(g, p, np.array([1.0]))["slp"][0]
    x = sgn * q
    assert u == pytest.approx((1 - x ** (p + 1)) / (1 - x) / (FOURPI * R), rel=1e-14)


def test_closed_form_legendre_terms(rng):
    """p = 3 written with explicit P_0..P_3 (textbook polynomials)."""
    for _ in range(10):
        c = rng.standard_normal(3)
        s = c + rng.standard_normal(3)
        t = c + 0.6 * np.linalg.norm(s - c) * rng.standard_normal(3) / np.sqrt(3) * 0.5
        R, rho = np.linalg.norm(s - c), np.linalg.norm(t - c)
        x = (t - c) @ (s - c) / (R * rho)
        P = [1, x, (3 * x * x - 1) / 2, (5 * x ** 3 - 3 * x) / 2]
        ref = sum(rho ** n / R ** (n + 1) * P[n] for n in range(4)) / FOURPI
        g = single_pair(t, c, s, w=2.0)
        assert oracle.tsqbx_laplace(g, 3, np.array([0.5]))["slp"][0] == pytest.approx(ref, rel=1e-14)


# -------------------------------------------------- convergence to kernels

def test_laplace_tail_bound_and_rate(rng):
    """|G - G^(p)| <= q^{p+1} / ((1-q) 4 pi R) with q = rho/R (|P_n| <= 1 in
    eq. laplace-potential-expansion); the error decays like q^{p+1}."""
    for _ in range(6):
        c = rng.standard_normal(3)
        s = c + rng.standard_normal(3)
        R = np.linalg.norm(s - c)
        q = rng.uniform(0.2, 0.7)
        dvec = rng.standard_normal(3)
        t = c + q * R * dvec / np.linalg.norm(dvec)
        g = single_pair(t, c, s)
        exact = oracle.point_potential(g, "laplace", np.array([1.0]))["slp"][0]
        assert exact == pytest.approx(1 / (FOURPI * np.linalg.norm(t - s)), rel=1e-15)
        errs = []
        for p in range(0, 41, 4):
            u = oracle.tsqbx_laplace(g, p, np.array([1.0]))["slp"][0]
            bound = q ** (p + 1) / ((1 - q) * FOURPI * R)
            assert abs(u - exact) <= bound * (1 + 1e-9) + 1e-16
            errs.append(abs(u - exact))
        assert errs[-1] < 1e-15 / R + q ** 41 / ((1 - q) * FOURPI * R)


def test_laplace_list_sums_converge(rng):
    g = cloud_geometry(rng, n_ctr=4, n_src=30, q_max=0.4, tgt_per_ctr=2)
    mu = rng.standard_normal(g.n_src)
    ref = oracle.point_potential(g, "laplace", mu, slp=True, dlp=True, sp=True)
    got = oracle.tsqbx_laplace(g, 40, mu, slp=True, dlp=True, sp=True)
    for k in ("slp", "dlp", "sp"):
        assert rel(got[k], ref[k]) < 1e-11, k
    # coarse p is visibly not converged (the test can fail)
    assert rel(oracle.tsqbx_laplace(g, 2, mu)["slp"], ref["slp"]) > 1e-6


def test_helmholtz_converges_and_k_to_zero(rng):
    g = cloud_geometry(rng, n_ctr=3, n_src=20, q_max=0.5, tgt_per_ctr=2)
    mu = rng.standard_normal(g.n_src) + 1j * rng.standard_normal(g.n_src)
    for k in (0.7, 4.0):
        ref = oracle.point_potential(g, "helmholtz", mu, k=k, slp=True, dlp=True, sp=True)
        got = oracle.tsqbx_helmholtz(g, 40, k, mu, slp=True, dlp=True, sp=True)
        for key in ("slp", "dlp", "sp"):
            assert rel(got[key], ref[key]) < 1e-10, (k, key)
    # k -> 0: ik (2n+1) j_n(k rho) h_n(kR) -> rho^n / R^{n+1}
    lap = oracle.tsqbx_laplace(g, 8, mu.real, slp=True, dlp=True, sp=True)
    hel = oracle.tsqbx_helmholtz(g, 8, 1e-5, mu.real.astype(complex), slp=True, dlp=True, sp=True)
    for key in ("slp", "dlp", "sp"):
        assert rel(hel[key].real, lap[key]) < 1e-8, key


# ----------------------------------------------- normal derivatives by FD

def test_normal_derivatives_match_finite_differences(rng):
    """DLP = d/deps of the SLP kernel at s + eps n_s; S' = d/deps at t + eps n_t."""
    c = np.array([0.2, 0.1, -0.3])
    s = c + np.array([0.7, -0.4, 0.5])
    t = c + np.array([0.1, 0.2, -0.15])
    ns = np.array([0.3, 0.9, -0.2]); ns /= np.linalg.norm(ns)
    nt = np.array([-0.5, 0.1, 0.8]); nt /= np.linalg.norm(nt)
    h = 1e-5
    for p in (0, 3, 9):
        g = single_pair(t, c, s, n_s=ns, n_t=nt)
        u = oracle.tsqbx_laplace(g, p, np.array([1.0]), slp=True, dlp=True, sp=True)
        f = lambda tt, ss: oracle.tsqbx_laplace(single_pair(tt, c, ss), p, np.array([1.0]))["slp"][0]
        fd_s = (f(t, s + h * ns) - f(t, s - h * ns)) / (2 * h)
        fd_t = (f(t + h * nt, s) - f(t - h * nt, s)) / (2 * h)
        assert u["dlp"][0] == pytest.approx(fd_s, rel=1e-8)
        assert u["sp"][0] == pytest.approx(fd_t, rel=1e-8)
        k = 3.0
        uh = oracle.tsqbx_helmholtz(g, p, k, np.array([1.0 + 0j]), slp=True, dlp=True, sp=True)
        fh = lambda tt, ss: oracle.tsqbx_helmholtz(single_pair(tt, c, ss), p, k,
                                                   np.array([1.0 + 0j]))["slp"][0]
        fd_s = (fh(t, s + h * ns) - fh(t, s - h * ns)) / (2 * h)
        fd_t = (fh(t + h * nt, s) - fh(t - h * nt, s)) / (2 * h)
        assert abs(uh["dlp"][0] - fd_s) <= 1e-8 * abs(fd_s)
        assert abs(uh["sp"][0] - fd_t) <= 1e-8 * abs(fd_t)


def test_target_normal_derivative_at_center_by_finite_differences():
    """S' at t = c (rho = 0, where that = (t-c)/|t-c| is undefined) equals the
    central difference of the SLP expansion through the center along n_t."""
    c = np.array([0.3, -0.1, 0.2])
    s = c + np.array([0.5, 0.6, -0.3])
    nt = np.array([0.2, -0.7, 0.4]); nt /= np.linalg.norm(nt)
    h = 1e-5
    for p in (1, 4, 9):
        g = single_pair(c, c, s, n_t=nt)
        u = oracle.tsqbx_laplace(g, p, np.array([1.0]), slp=True, sp=True)
        f = lambda tt: oracle.tsqbx_laplace(single_pair(tt, c, s), p, np.array([1.0]))["slp"][0]
        assert u["sp"][0] == pytest.approx((f(c + h * nt) - f(c - h * nt)) / (2 * h), rel=1e-8)
        for k in (0.8, 6.0):
            uh = oracle.tsqbx_helmholtz(g, p, k, np.array([1.0 + 0j]), sp=True)["sp"][0]
            fh = lambda tt: oracle.tsqbx_helmholtz(single_pair(tt, c, s), p, k,
                                                   np.array([1.0 + 0j]))["slp"][0]
            fd = (fh(c + h * nt) - fh(c - h * nt)) / (2 * h)
            assert abs(uh - fd) <= 1e-8 * abs(fd)


def test_conventional_path_target_derivative_at_center_by_finite_differences():
    """Path B on its own: S' at t = c equals the central difference of path
    B's single layer through the center along n_t (Laplace and Helmholtz)."""
    c = np.array([-0.2, 0.4, 0.1])
    s = c + np.array([-0.4, 0.5, 0.6])
    nt = np.array([0.6, 0.3, -0.7]); nt /= np.linalg.norm(nt)
    h = 1e-5
    for p in (1, 3, 8):
        g = single_pair(c, c, s, n_t=nt)
        u = oracle.qbx_laplace(g, p, np.array([1.0]), slp=True, sp=True)["sp"][0]
        f = lambda tt: oracle.qbx_laplace(single_pair(tt, c, s), p, np.array([1.0]))["slp"][0]
        assert u == pytest.approx((f(c + h * nt) - f(c - h * nt)) / (2 * h), rel=1e-8)
        for k in (0.7, 5.0):
            uh = oracle.qbx_helmholtz(g, p, k, np.array([1.0 + 0j]), sp=True)["sp"][0]
            fh = lambda tt: oracle.qbx_helmholtz(single_pair(tt, c, s), p, k,
                                                 np.array([1.0 + 0j]))["slp"][0]
            fd = (fh(c + h * nt) - fh(c - h * nt)) / (2 * h)
            assert abs(uh - fd) <= 1e-8 * abs(fd)


# ------------------------------------------------- 50-digit brute force

def _mp_laplace(t, c, s, ns, p):
    with mpmath.workdps(50):
        T = [mpmath.mpf(v) for v in t]
        C = [mpmath.mpf(v) for v in c]
        S = [mpmath.mpf(v) for v in s]
        N = [mpmath.mpf(v) for v in ns]
        tc = [a - b for a, b in zip(T, C)]
        sc = [a - b for a, b in zip(S, C)]
        rho = mpmath.sqrt(sum(v * v for v in tc))
        R = mpmath.sqrt(sum(v * v for v in sc))
        x = sum(a * b for a, b in zip(tc, sc)) / (rho * R)
        slp = sum(rho ** n / R ** (n + 1) * mpmath.legendre(n, x) for n in range(p + 1))
        shn = sum(a * b for a, b in zip(sc, N)) / R
        thn = sum(a * b for a, b in zip(tc, N)) / rho
        dlp = 0
        for n in range(p + 1):
            dPn = mpmath.diff(lambda u: mpmath.legendre(n, u), x)
            dlp += rho ** n / R ** (n + 2) * (-(n + 1) * shn * mpmath.legendre(n, x)
                                              + (thn - shn * x) * dPn)
        return float(slp / (4 * mpmath.pi)), float(dlp / (4 * mpmath.pi))


def _mp_helmholtz(t, c, s, p, k):
    with mpmath.workdps(50):
        T = [mpmath.mpf(v) for v in t]
        C = [mpmath.mpf(v) for v in c]
        S = [mpmath.mpf(v) for v in s]
        K = mpmath.mpf(k)
        tc = [a - b for a, b in zip(T, C)]
        sc = [a - b for a, b in zip(S, C)]
        rho = mpmath.sqrt(sum(v * v for v in tc))
        R = mpmath.sqrt(sum(v * v for v in sc))
        x = sum(a * b for a, b in zip(tc, sc)) / (rho * R)

        def sj(n, z):
            return mpmath.sqrt(mpmath.pi / (2 * z)) * mpmath.besselj(n + mpmath.mpf(1) / 2, z)

        def sy(n, z):
            return mpmath.sqrt(mpmath.pi / (2 * z)) * mpmath.bessely(n + mpmath.mpf(1) / 2, z)

        acc = 0
        for n in range(p + 1):
            h = sj(n, K * R) + 1j * sy(n, K * R)
            acc += (2 * n + 1) * sj(n, K * rho) * h * mpmath.legendre(n, x)
        v = 1j * K / (4 * mpmath.pi) * acc
        return complex(v)


def test_brute_force_tiny_cases(rng):
    for _ in range(12):
        c = rng.uniform(-1, 1, 3)
        s = c + rng.standard_normal(3)
        R = np.linalg.norm(s - c)
        d = rng.standard_normal(3)
        t = c + rng.uniform(0.1, 0.9) * R * d / np.linalg.norm(d)
        ns = rng.standard_normal(3); ns /= np.linalg.norm(ns)
        p = int(rng.integers(0, 13))
        g = single_pair(t, c, s, n_s=ns)
        u = oracle.tsqbx_laplace(g, p, np.array([1.0]), slp=True, dlp=True)
        slp, dlp = _mp_laplace(t, c, s, ns, p)
        assert u["slp"][0] == pytest.approx(slp, rel=1e-13)
        assert u["dlp"][0] == pytest.approx(dlp, rel=1e-11, abs=1e-13 * abs(slp))
        k = float(rng.uniform(0.5, 10))
        uh = oracle.tsqbx_helmholtz(g, p, k, np.array([1.0 + 0j]))["slp"][0]
        ref = _mp_helmholtz(t, c, s, p, k)
        assert abs(uh - ref) <= 1e-12 * abs(ref)


def _select_ranges(g, keep):
    """Same geometry with each group's ranges filtered by keep(group, i, n)."""
    import copy
    grs, rb, re = [0], [], []
    for q in range(g.n_group):
        a, b = g.group_range_start[q], g.group_range_start[q + 1]
        for i in range(a, b):
            if keep(q, i - a, b - a):
                rb.append(g.range_begin[i]); re.append(g.range_end[i])
        grs.append(len(rb))
    h = copy.copy(g)
    h.group_range_start = np.array(grs, np.int64)
    h.range_begin = np.array(rb, np.int32)
    h.range_end = np.array(re, np.int32)
    return h


def test_duplicate_ranges_are_summed_twice(rng):
    """A range listed twice contributes twice: u(all) = u(all but last) + u(last)."""
    g = cloud_geometry(rng, n_ctr=3, n_src=20, dup=True)
    mu = rng.standard_normal(g.n_src)
    u = oracle.tsqbx_laplace(g, 4, mu)["slp"]
    head = oracle.tsqbx_laplace(_select_ranges(g, lambda q, i, n: i < n - 1), 4, mu)["slp"]
    tail = oracle.tsqbx_laplace(_select_ranges(g, lambda q, i, n: i == n - 1), 4, mu)["slp"]
    np.testing.assert_allclose(u, head + tail, rtol=1e-13)
    n = oracle.count_pairs(g)
    lens = g.range_end - g.range_begin
    per_group = [lens[g.group_range_start[q]:g.group_range_start[q + 1]].sum()
                 for q in range(g.n_group)]
    assert n == sum(per_group[g.ctr_group[g.tgt_center[t]]] for t in range(g.n_tgt))
