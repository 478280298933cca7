"""The constants the kernels take from their headers, read through a test
shim (tests/native/constants_shim.cu) and checked in 30-digit arithmetic:

* the scaled Legendre recurrences: kappa_n = (2n-1)!!/n! and beta_n with
  Q_n = kappa_n T_n, and lambda_n, gamma_n with Q'_n = lambda_n U_n;
* the conventional Laplace path: with the irregular and regular solid
  harmonics J_n^m, K_n^m built by the recurrences its header states (eps_n^m
  from the library), the weights w_n^m give
  sum_m w_n^m Re(K_n^m(e) conj J_n^m(d)) = |e|^n / |d|^{n+1} P_n(cos g) / (4 pi)
  for every n <= 20 (eq. legendre-addition-identity);
* the conventional Helmholtz path: omega_n^m = 4 pi kappa_n times its weights
  gives sum_m omega_n^m (Re J(v) Re J(u) + Im J(v) Im J(u)) = P_n(u.v) for
  unit u, v and every n up to its largest order.
"""
import ctypes

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 30


@pytest.fixture(scope="module")
def K():
    from helpers import native_shim
    path = native_shim("constants_shim")
    if path is None:
        pytest.skip("no nvcc")
    L = ctypes.CDLL(path)
    for name in ("shim_rec_kappa", "shim_rec_beta", "shim_rec_lambda", "shim_rec_gamma"):
        getattr(L, name).argtypes = [ctypes.c_int]
        getattr(L, name).restype = ctypes.c_double
    for name in ("shim_conv_eps", "shim_conv_weight", "shim_conv_helm_weight"):
        getattr(L, name).argtypes = [ctypes.c_int, ctypes.c_int]
        getattr(L, name).restype = ctypes.c_double
    L.shim_inv_4pi.restype = ctypes.c_double
    return L


def _rel(a, b):
    return abs(a - b) / max(abs(b), mpmath.mpf(10) ** -300)


def test_scaled_recurrence_constants(K):
    assert _rel(mpmath.mpf(K.shim_inv_4pi()), 1 / (4 * mpmath.pi)) < 1e-16
    for n in range(0, 22):
        assert _rel(mpmath.mpf(K.shim_rec_kappa(n)), mpmath.fac2(2 * n - 1) / mpmath.factorial(n)) < 1e-15
        if n >= 1:
            assert _rel(mpmath.mpf(K.shim_rec_beta(n)), mpmath.mpf(n * n) / ((2 * n + 1) * (2 * n - 1))) < 1e-15
            assert abs(mpmath.mpf(K.shim_rec_gamma(n)) - mpmath.mpf(n * n - 1) / (4 * n * n - 1)) < 1e-16
    # Q'_n = lambda_n U_n with U_{n+1} = qx U_n - gamma_n q2 U_{n-1}, U_0 = 0, U_1 = 1
    rng = np.random.default_rng(2)
    for _ in range(4):
        r = mpmath.mpf(float(rng.uniform(0.1, 0.9)))
        x = mpmath.mpf(float(rng.uniform(-1, 1)))
        qx, q2 = r * x, r * r
        U = [mpmath.mpf(0), mpmath.mpf(1)]
        for n in range(1, 21):
            U.append(qx * U[n] - mpmath.mpf(K.shim_rec_gamma(n)) * q2 * U[n - 1])
        for n in range(1, 22):
            want = r ** (n - 1) * mpmath.diff(lambda y: mpmath.legendre(n, y), x)
            assert abs(mpmath.mpf(K.shim_rec_lambda(n)) * U[n] - want) < 1e-13 * max(abs(want), 1)


def _solid_harmonics(K, v, p, irregular):
    """J_n^m (irregular, 1/r^(n+1)) or K_n^m (regular, r^n) for 0 <= m <= n <= p
    by the recurrences of the conventional path's header."""
    x, y, z = v
    r2 = x * x + y * y + z * z
    if irregular:
        a = 1 / r2
        lead, step, sq = mpmath.sqrt(a), (x + 1j * y) * a, a          # J_0^0 = 1/r, eta, a
        zeta = z * a
    else:
        lead, step, sq = mpmath.mpf(1), x + 1j * y, r2                # K_0^0 = 1, xi, r^2
        zeta = z
    H = {}
    diag = lead
    for m in range(p + 1):
        if m > 0:
            diag = step * diag
        H[(m, m)] = diag
        if m + 1 <= p:
            H[(m + 1, m)] = zeta * diag
        for n in range(m + 2, p + 1):
            H[(n, m)] = zeta * H[(n - 1, m)] - mpmath.mpf(K.shim_conv_eps(n, m)) * sq * H[(n - 2, m)]
    return H


@pytest.mark.parametrize("seed", range(3))
def test_laplace_conventional_weights_give_the_addition_theorem(K, seed):
    rng = np.random.default_rng(seed)
    d = [mpmath.mpf(float(v)) for v in rng.standard_normal(3)]
    e = [mpmath.mpf(float(v)) for v in 0.5 * rng.standard_normal(3)]
    p = 20
    J = _solid_harmonics(K, d, p, True)
    Kh = _solid_harmonics(K, e, p, False)
    R = mpmath.sqrt(sum(v * v for v in d))
    rho = mpmath.sqrt(sum(v * v for v in e))
    cosg = sum(a * b for a, b in zip(d, e)) / (R * rho)
    for n in range(p + 1):
        s = sum(mpmath.mpf(K.shim_conv_weight(n, m)) * mpmath.re(Kh[(n, m)] * mpmath.conj(J[(n, m)]))
                for m in range(n + 1))
        want = rho ** n / R ** (n + 1) * mpmath.legendre(n, cosg) / (4 * mpmath.pi)
        assert abs(s - want) <= 1e-13 * rho ** n / R ** (n + 1), n


@pytest.mark.parametrize("seed", range(3))
def test_helmholtz_conventional_weights_give_the_addition_theorem(K, seed):
    rng = np.random.default_rng(10 + seed)
    u = rng.standard_normal(3)
    v = rng.standard_normal(3)
    u = [mpmath.mpf(float(c)) for c in u / np.linalg.norm(u)]
    v = [mpmath.mpf(float(c)) for c in v / np.linalg.norm(v)]
    p = K.shim_conv_helm_max_p()
    assert p >= 12
    # the angular harmonics at unit radius: the irregular recurrence with a = 1
    Ju = _solid_harmonics(K, u, p, True)
    Jv = _solid_harmonics(K, v, p, True)
    nu = mpmath.sqrt(sum(c * c for c in u))
    cosg = sum(a * b for a, b in zip(u, v)) / (nu * mpmath.sqrt(sum(c * c for c in v)))
    for n in range(p + 1):
        omega = [4 * mpmath.pi * mpmath.mpf(K.shim_rec_kappa(n)) * mpmath.mpf(K.shim_conv_helm_weight(n, m))
                 for m in range(n + 1)]
        want_omega = [(1 if m == 0 else 2) * mpmath.fac2(2 * n - 1) ** 2
                      / (mpmath.factorial(n + m) * mpmath.factorial(n - m)) for m in range(n + 1)]
        for m in range(n + 1):
            assert _rel(omega[m], want_omega[m]) < 1e-14
        s = sum(omega[m] * (mpmath.re(Jv[(n, m)]) * mpmath.re(Ju[(n, m)])
                            + mpmath.im(Jv[(n, m)]) * mpmath.im(Ju[(n, m)])) for m in range(n + 1))
        assert abs(s - mpmath.legendre(n, cosg)) < 1e-12, n


def test_double_float_constants(K):
    """df_const splits a double constant into floats hi + lo with hi the
    nearest float and |lo| <= ulp(hi)/2, so that hi + lo carries it to about
    2^-48 relative: the form the double-float kernel takes kappa_n, beta_n,
    the Gegenbauer constants and 1/(4 pi) in."""
    K.shim_df_const.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    hi, lo = ctypes.c_float(), ctypes.c_float()
    values = [K.shim_inv_4pi()] + [K.shim_rec_kappa(n) for n in range(21)] + \
             [K.shim_rec_beta(n) for n in range(1, 22)] + [K.shim_rec_gamma(n) for n in range(2, 22)] + \
             [K.shim_rec_lambda(n) for n in range(1, 22)]
    for v in values:
        K.shim_df_const(v, ctypes.byref(hi), ctypes.byref(lo))
        assert hi.value == float(np.float32(v))
        assert abs(lo.value) <= np.spacing(np.float32(abs(hi.value))) / 2
        assert abs((float(hi.value) + float(lo.value)) - v) <= 2.0 ** -48 * abs(v)
