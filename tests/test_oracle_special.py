"""Pins for the oracle's special functions (Legendre, spherical Bessel/Hankel,
spherical harmonics) against closed forms, identities and library routines."""
import numpy as np
import pytest
import scipy.special as sp

import oracle

mpmath = pytest.importorskip("mpmath")


@pytest.mark.parametrize("x", [-1.0, -0.73, -0.2, 0.0, 0.31, 0.9, 1.0])
def test_legendre_closed_forms(x):
    P, dP = oracle.legendre(3, x)
    assert P[0] == 1.0 and P[1] == x
    assert P[2] == pytest.approx((3 * x * x - 1) / 2, abs=1e-15)
    assert P[3] == pytest.approx((5 * x ** 3 - 3 * x) / 2, abs=1e-15)
    assert dP[0] == 0.0 and dP[1] == 1.0
    assert dP[2] == pytest.approx(3 * x, abs=1e-15)
    assert dP[3] == pytest.approx((15 * x * x - 3) / 2, abs=1e-14)


def test_legendre_against_scipy_and_endpoints():
    for x in np.linspace(-1, 1, 41):
        P, dP = oracle.legendre(30, x)
        ref = np.array([sp.eval_legendre(n, x) for n in range(31)])
        np.testing.assert_allclose(P, ref, atol=1e-13)
        with mpmath.workdps(40):
            for n in range(1, 21):
                dref = float(mpmath.diff(lambda u: mpmath.legendre(n, u), mpmath.mpf(x)))
                assert dP[n] == pytest.approx(dref, rel=1e-12, abs=1e-12)
    for s in (1.0, -1.0):
        P, dP = oracle.legendre(25, s)
        n = np.arange(26)
        np.testing.assert_array_equal(P, s ** n)
        np.testing.assert_allclose(dP, s ** (n + 1) * n * (n + 1) / 2, rtol=1e-14)


@pytest.mark.parametrize("z", [1e-3, 0.05, 0.3, 1.0, 2.5, 7.0, 15.0, 40.0])
def test_spherical_bessel_closed_forms(z):
    """DLMF 10.49.3 / 10.49.4 for n <= 2, evaluated at 50 digits (the closed
    forms cancel badly at small z in double precision)."""
    j, y = oracle.sph_jn(2, z), oracle.sph_yn(2, z)
    with mpmath.workdps(50):
        Z = mpmath.mpf(z)
        s, c = mpmath.sin(Z), mpmath.cos(Z)
        jref = [s / Z, s / Z ** 2 - c / Z, (3 / Z ** 2 - 1) * s / Z - 3 * c / Z ** 2]
        yref = [-c / Z, -c / Z ** 2 - s / Z, (-3 / Z ** 2 + 1) * c / Z - 3 * s / Z ** 2]
        jref = [float(v) for v in jref]
        yref = [float(v) for v in yref]
    for n in range(3):
        assert j[n] == pytest.approx(jref[n], rel=1e-12)
        assert y[n] == pytest.approx(yref[n], rel=1e-12)


@pytest.mark.parametrize("z", [1e-2, 0.1, 0.7, 1.9, 4.4, 9.5, 20.0])
def test_spherical_bessel_against_scipy_and_wronskian(z):
    nmax = 24
    j, y = oracle.sph_jn(nmax, z), oracle.sph_yn(nmax, z)
    n = np.arange(nmax + 1)
    np.testing.assert_allclose(j, sp.spherical_jn(n, z), rtol=1e-11, atol=1e-300)
    np.testing.assert_allclose(y, sp.spherical_yn(n, z), rtol=1e-11)
    # Wronskian, DLMF 10.50.3: j_{n+1} y_n - j_n y_{n+1} = 1/z^2
    w = j[1:] * y[:-1] - j[:-1] * y[1:]
    np.testing.assert_allclose(w * z * z, np.ones(nmax), rtol=1e-10)
    dj, dy = oracle.sph_jn_deriv(nmax - 1, z), oracle.sph_yn_deriv(nmax - 1, z)
    m = np.arange(nmax)
    np.testing.assert_allclose(dj, sp.spherical_jn(m, z, derivative=True), rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(dy, sp.spherical_yn(m, z, derivative=True), rtol=1e-10)


def test_jn_at_zero():
    j = oracle.sph_jn(5, 0.0)
    np.testing.assert_array_equal(j, [1, 0, 0, 0, 0, 0])


def test_sph_harm_against_scipy(rng):
    """eq. sph-harm without the Condon-Shortley phase: Y_n^m = (-1)^m Y_scipy for
    m >= 0 and = Y_scipy for m < 0 (scipy includes the phase in P_n^m)."""
    p = 8
    for v in rng.standard_normal((10, 3)):
        Y = oracle.sph_harm(p, v)
        r = np.linalg.norm(v)
        theta, phi = np.arccos(v[2] / r), np.arctan2(v[1], v[0])
        for n in range(p + 1):
            for m in range(-n, n + 1):
                ref = sp.sph_harm_y(n, m, theta, phi)
                if m >= 0:
                    ref = ref * (-1) ** m
                assert Y[n * n + n + m] == pytest.approx(ref, abs=1e-13)


def test_legendre_addition_identity(rng):
    """eq. legendre-addition-identity: P_n(cos g) = 4 pi/(2n+1) sum_m Y_n^m(a) Y_n^-m(b)."""
    p = 10
    for _ in range(5):
        a, b = rng.standard_normal(3), rng.standard_normal(3)
        Ya, Yb = oracle.sph_harm(p, a), oracle.sph_harm(p, b)
        x = a @ b / np.linalg.norm(a) / np.linalg.norm(b)
        for n in range(p + 1):
            s = sum(Ya[n * n + n + m] * Yb[n * n + n - m] for m in range(-n, n + 1))
            assert s.imag == pytest.approx(0.0, abs=1e-13)
            assert 4 * np.pi / (2 * n + 1) * s.real == pytest.approx(sp.eval_legendre(n, x), abs=1e-13)


def test_oracle_rejects_invalid_lists_and_orders():
    """The oracle checks its inputs instead of reading out of bounds: ranges
    past the sources, targets mapped to missing centers, orders out of range
    and a non-positive wavenumber are refused."""
    from helpers import cloud_geometry
    rng = np.random.default_rng(21)
    g = cloud_geometry(rng, n_ctr=3, n_src=30)
    mu = rng.standard_normal(g.n_src)
    oracle.tsqbx_laplace(g, 4, mu)                       # valid input runs
    for mutate in (lambda h: setattr(h, "range_end", h.range_end + 100),
                   lambda h: setattr(h, "tgt_center", np.full_like(h.tgt_center, 7)),
                   lambda h: setattr(h, "ctr_group", np.full_like(h.ctr_group, -1))):
        h = cloud_geometry(np.random.default_rng(21), n_ctr=3, n_src=30)
        mutate(h)
        with pytest.raises(ValueError):
            oracle.tsqbx_laplace(h, 4, mu)
    with pytest.raises(ValueError):
        oracle.tsqbx_laplace(g, -1, mu)
    with pytest.raises(ValueError):
        oracle.tsqbx_laplace(g, 41, mu)
    with pytest.raises(ValueError):
        oracle.tsqbx_helmholtz(g, 4, 0.0, mu.astype(complex))
