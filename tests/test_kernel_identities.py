"""The identities the GPU kernels' summation forms rest on, checked in 40-digit
arithmetic against the textbook functions (mpmath), independently of both
the oracle and the kernels.

Laplace (Appendix A with x = cos g, qx = (rho/R) x, q2 = (rho/R)^2,
Q_n = (rho/R)^n P_n(x), Q'_n = (rho/R)^(n-1) P'_n(x)):
  * Q_n = kappa_n T_n with kappa_n = (2n-1)!!/n!, T_{n+1} = qx T_n - beta_n q2 T_{n-1},
    beta_n = n^2/((2n+1)(2n-1)), and Clenshaw's backward sum of kappa_n T_n;
  * n Q'_{n+1} = (2n+1) qx Q'_n - (n+1) q2 Q'_{n-1} (Gegenbauer C^(3/2));
  * sum Q_n = (1 - 2 qx + q2) sum Q'_n + Q'_{p+1} - q2 Q'_p and
    sum (n+1) Q_n = (1 - qx) sum Q'_n + Q'_{p+1};
  * the double layer and S' written with these sums equal the Appendix A
    gradients term by term.
Helmholtz (h_n = h_n^(1), z = kR):
  * h_n(z) = e^{iz} g_n(z), g_0 = -i/z, g_1 = -(1/z + i/z^2), and g_n obeys
    f_{n+1} = (2n+1)/z f_n - f_{n-1} (DLMF 10.51.1), with g_{-1} = 1/z;
  * Clenshaw over g_n: sum c_n g_n = (c_0 - b_2) g_0 + b_1 g_1 for real c_n;
  * sum a_n (g_{n-1} - (n+1)/z g_n) = a_0/z + sum (a_{n+1} - (n+1)/z a_n) g_n.
"""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp
mp.dps = 40

TOL = mpmath.mpf(10) ** -30


def _close(a, b, scale=None):
    s = scale if scale is not None else max(abs(b), mpmath.mpf(1))
    return abs(a - b) <= TOL * s


def _geometry(rng):
    """d = s - c, e = t - c with |e| < 0.9 |d|, unit normals."""
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    d *= rng.uniform(0.5, 2.0)
    e = rng.standard_normal(3)
    e *= rng.uniform(0.05, 0.9) * np.linalg.norm(d) / np.linalg.norm(e)
    ns = rng.standard_normal(3)
    nt = rng.standard_normal(3)
    return ([mpmath.mpf(float(v)) for v in d], [mpmath.mpf(float(v)) for v in e],
            [mpmath.mpf(float(v)) for v in ns / np.linalg.norm(ns)],
            [mpmath.mpf(float(v)) for v in nt / np.linalg.norm(nt)])


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def _P(n, x):
    return mpmath.legendre(n, x)


def _dP(n, x):
    return mpmath.diff(lambda y: mpmath.legendre(n, y), x)


@pytest.mark.parametrize("seed", range(6))
def test_laplace_scaled_bonnet_and_clenshaw(seed):
    d, e, _, _ = _geometry(np.random.default_rng(seed))
    R2, rho2 = _dot(d, d), _dot(e, e)
    qx, q2 = _dot(d, e) / R2, rho2 / R2
    x = _dot(d, e) / mpmath.sqrt(R2 * rho2)
    r = mpmath.sqrt(q2)
    for p in (0, 1, 5, 9, 20):
        kappa = [mpmath.fac2(2 * n - 1) / mpmath.factorial(n) for n in range(p + 1)]
        beta = [mpmath.mpf(n * n) / ((2 * n + 1) * (2 * n - 1)) for n in range(p + 2)]
        T = [mpmath.mpf(1), qx]
        for n in range(1, p):
            T.append(qx * T[n] - beta[n] * q2 * T[n - 1])
        for n in range(p + 1):
            assert _close(kappa[n] * T[n], r ** n * _P(n, x))
        b = [mpmath.mpf(0)] * (p + 3)
        for k in range(p, -1, -1):
            b[k] = kappa[k] + qx * b[k + 1] - beta[k + 1] * q2 * b[k + 2]
        assert _close(b[0], sum(r ** n * _P(n, x) for n in range(p + 1)))


@pytest.mark.parametrize("seed", range(6))
def test_laplace_derivative_recurrence_and_closing_sums(seed):
    d, e, _, _ = _geometry(np.random.default_rng(seed))
    R2, rho2 = _dot(d, d), _dot(e, e)
    qx, q2 = _dot(d, e) / R2, rho2 / R2
    x = _dot(d, e) / mpmath.sqrt(R2 * rho2)
    r = mpmath.sqrt(q2)
    pmax = 21
    Qp = [mpmath.mpf(0), mpmath.mpf(1)]                        # Q'_0, Q'_1
    for n in range(1, pmax):
        Qp.append(((2 * n + 1) * qx * Qp[n] - (n + 1) * q2 * Qp[n - 1]) / n)
    for n in range(1, pmax + 1):
        assert _close(Qp[n], r ** (n - 1) * _dP(n, x))
    for p in (0, 1, 5, 9, 20):
        Q = [r ** n * _P(n, x) for n in range(p + 1)]
        SQp = sum(Qp[: p + 1])
        assert _close(sum(Q), (1 - 2 * qx + q2) * SQp + Qp[p + 1] - q2 * Qp[p])
        assert _close(sum((n + 1) * Q[n] for n in range(p + 1)), (1 - qx) * SQp + Qp[p + 1])


@pytest.mark.parametrize("seed", range(6))
def test_laplace_layer_closures_equal_appendix_a_gradients(seed):
    """DLP = [(b - a) sum Q'_n - a Q'_{p+1}] / (4 pi R^3), a = d.n_s, b = e.n_s;
    S' = [(d.n_t) sum_{n<=p} Q'_n - (e.n_t) sum_{n<p} Q'_n] / (4 pi R^3)."""
    d, e, ns, nt = _geometry(np.random.default_rng(100 + seed))
    R2, rho2 = _dot(d, d), _dot(e, e)
    R, rho = mpmath.sqrt(R2), mpmath.sqrt(rho2)
    qx, q2 = _dot(d, e) / R2, rho2 / R2
    x = _dot(d, e) / (R * rho)
    shat = [v / R for v in d]
    that = [v / rho for v in e]
    Qp = [mpmath.mpf(0), mpmath.mpf(1)]
    for n in range(1, 21):
        Qp.append(((2 * n + 1) * qx * Qp[n] - (n + 1) * q2 * Qp[n - 1]) / n)
    four_pi = 4 * mpmath.pi
    for p in (0, 1, 4, 9, 20):
        # Appendix A: n_s.grad_s and n_t.grad_t of G^(p)
        dlp = sum(rho ** n / R ** (n + 2) * (-(n + 1) * _dot(shat, ns) * _P(n, x)
                                             + (_dot(that, ns) - x * _dot(shat, ns)) * _dP(n, x))
                  for n in range(p + 1)) / four_pi
        sp = sum(rho ** (n - 1) / R ** (n + 1) * (n * _dot(that, nt) * _P(n, x)
                                                  + (_dot(shat, nt) - x * _dot(that, nt)) * _dP(n, x))
                 for n in range(1, p + 1)) / four_pi
        a, b = _dot(d, ns), _dot(e, ns)
        dlp_k = ((b - a) * sum(Qp[: p + 1]) - a * Qp[p + 1]) / (four_pi * R ** 3)
        sp_k = (_dot(d, nt) * sum(Qp[: p + 1]) - _dot(e, nt) * sum(Qp[:p])) / (four_pi * R ** 3)
        assert _close(dlp_k, dlp, abs(dlp) + 1 / R ** 2)
        assert _close(sp_k, sp, abs(sp) + 1 / R ** 2)


def _h(n, z):
    f = mpmath.sqrt(mpmath.pi / (2 * z))
    return f * (mpmath.besselj(n + mpmath.mpf(1) / 2, z) + 1j * mpmath.bessely(n + mpmath.mpf(1) / 2, z))


@pytest.mark.parametrize("z", ["0.01", "0.7", "3.0", "25.0", "100.0"])
def test_hankel_factor_recurrence(z):
    z = mpmath.mpf(z)
    g = [-1j / z, -(1 / z + 1j / z ** 2)]
    for n in range(1, 20):
        g.append((2 * n + 1) / z * g[n] - g[n - 1])
    e = mpmath.exp(1j * z)
    for n in range(21):
        assert _close(e * g[n], _h(n, z), abs(_h(n, z)))
    # the n = 0 step gives g_{-1} = 1/z
    assert _close(g[0] / z - g[1], 1 / z)


@pytest.mark.parametrize("z", ["0.05", "2.0", "40.0"])
def test_clenshaw_over_hankel_factors(z):
    z = mpmath.mpf(z)
    rng = np.random.default_rng(int(float(z) * 100))
    p = 15
    g = [-1j / z, -(1 / z + 1j / z ** 2)]
    for n in range(1, p + 1):
        g.append((2 * n + 1) / z * g[n] - g[n - 1])
    c = [mpmath.mpf(float(v)) for v in rng.standard_normal(p + 1)]
    b = [mpmath.mpf(0)] * (p + 3)
    for n in range(p, -1, -1):
        b[n] = c[n] + (2 * n + 1) / z * b[n + 1] - b[n + 2]
    direct = sum(c[n] * g[n] for n in range(p + 1))
    assert _close((c[0] - b[2]) * g[0] + b[1] * g[1], direct, max(abs(t) for t in
                                                                  (c[n] * g[n] for n in range(p + 1))))
    # the double layer's derivative sum
    a = [mpmath.mpf(float(v)) for v in rng.standard_normal(p + 1)] + [mpmath.mpf(0)]
    gm1 = 1 / z
    lhs = sum(a[n] * ((g[n - 1] if n > 0 else gm1) - (n + 1) / z * g[n]) for n in range(p + 1))
    rhs = a[0] / z + sum((a[n + 1] - (n + 1) / z * a[n]) * g[n] for n in range(p + 1))
    assert _close(lhs, rhs, max(abs(lhs), max(abs(t) for t in g)))
