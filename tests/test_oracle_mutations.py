"""The pins are sensitive: plausible mistakes planted in copies of oracle.c
(a wrong sign, a dropped factor, an index off by one, transposed operands, the
wrong Hankel kind, a wrong derivative rule, a too-short recurrence) each make at
least one pin test fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "bonnet_sign": ("(2.0 * n + 1.0) * x * P[n] - n * P[n - 1]",
                    "(2.0 * n + 1.0) * x * P[n] + n * P[n - 1]"),
    "dP_index": ("x * dP[n] + (n + 1.0) * P[n]", "x * dP[n] + n * P[n]"),
    "slp_power": ("pow(pg.rho, n) / pow(pg.R, n + 1) * P[n]", "pow(pg.rho, n) / pow(pg.R, n) * P[n]"),
    "dlp_factor": ("-(n + 1.0) * shn * P[n]", "-(double)n * shn * P[n]"),
    "dlp_transposed": ("(thn - shn * pg.x) * dP[n]", "(shn - thn * pg.x) * dP[n]"),
    "sp_transposed": ("n * thn * P[n] + (shn - thn * pg.x)", "n * shn * P[n] + (shn - thn * pg.x)"),
    "hankel_kind": ("acc += (2.0 * n + 1.0) * jt[n] * (js[n] + I * ys[n]) * P[n];",
                    "acc += (2.0 * n + 1.0) * jt[n] * (js[n] - I * ys[n]) * P[n];"),
    "miller_norm": ("j0 / f[0] : j1 / f[1]", "j1 / f[0] : j0 / f[1]"),
    "yn_recurrence": ("y[n + 1] = (2.0 * n + 1.0) / z * y[n] - y[n - 1]",
                      "y[n + 1] = (2.0 * n - 1.0) / z * y[n] - y[n - 1]"),
    "hankel_deriv": ("(k * scn * dh * P[n] + tsn * h * dP[n])", "(k * scn * h * P[n] + tsn * h * dP[n])"),
    "pathB_conjugate": ("cdmul(f, Y[n * n + n - m])", "cdmul(f, Y[n * n + n + m])"),
    "four_pi": ("nsum_add(&us, wmu * nsum_get(&acc) / (4.0 * ORACLE_PI));",
                "nsum_add(&us, wmu * nsum_get(&acc) / (2.0 * ORACLE_PI));"),
    "sp_rho0_limit": ("acc = k * (js[1] + I * ys[1]) * dot3(pg.shat, nt_);",
                      "acc = (js[1] + I * ys[1]) * dot3(pg.shat, nt_);"),
    "pathB_sp_rho0_slope": ("const double slope = kernel == 0 ? 1.0 : k / 3.0;",
                            "const double slope = kernel == 0 ? 1.0 : k / 2.0;"),
    "helm_sp_no_derivative": ("(k * tcn * djt[n] * P[n] + stn * jt[n] * dP[n])",
                              "(k * tcn * jt[n] * P[n] + stn * jt[n] * dP[n])"),
    "helm_sp_transposed": ("dot3(pg.shat, nt_) - dot3(pg.that_, nt_) * pg.x",
                           "dot3(pg.that_, nt_) - dot3(pg.shat, nt_) * pg.x"),
    "pathB_helm_missing_i": ("double complex a = I * k * h, b", "double complex a = k * h, b"),
    "pathB_dual_chain": ("b = I * k * (k * R.d) * dh;", "b = I * k * R.d * dh;"),
    "pathB_laplace_2n1": ("dscale(Rpow, 2.0 * n + 1.0)", "dscale(Rpow, 2.0 * n + 2.0)"),
    "sph_harm_dual_recurrence": ("dual t2 = dscale(A[n - 1][m], (double)(n + m));",
                                 "dual t2 = dscale(A[n - 1][m], (double)(n - m));"),
    "dual_quotient_sign": ("(a.d * b.v - a.v * b.d) / (b.v * b.v)", "(a.d * b.v + a.v * b.d) / (b.v * b.v)"),
    "bessel_deriv_index": ("df[n] = f[n - 1] - (n + 1.0) / z * f[n];", "df[n] = f[n - 1] - n / z * f[n];"),
    "miller_short_start": ("int N = nmax + 20 + (int)ceil(z);", "int N = nmax + 1;"),
    "point_dlp_sign": ("wmu * dG * dot3(ns, ts), -wmu", "-wmu * dG * dot3(ns, ts), -wmu"),
    "point_helm_outgoing": ("e * (1.0 - I * k * rr)", "e * (1.0 + I * k * rr)"),
    "pathB_laplace_sp_slope": ("const double slope = kernel == 0 ? 1.0 : k / 3.0;",
                               "const double slope = kernel == 0 ? 0.5 : k / 3.0;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(scratch, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mut = scratch / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    lib = scratch / "liboracle_mut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(mut), "-o", str(lib), "-lm"],
                   check=True, capture_output=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_special.py"),
                        os.path.join(ROOT, "tests", "test_oracle_expansions.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught mutation {name}:\n{r.stdout[-2000:]}"
