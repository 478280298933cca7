/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the near-field target-specific
 * QBX (TSQBX) step of GIGAQBX (Wala & Kloeckner, arXiv:1811.01110).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline /
 * reference arm use it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (per target t with QBX center c, summed over every source s
 * listed in the center's group's half-open source ranges, duplicates included):
 *
 *  Path A -- the target-specific expansion written out as in Appendix A:
 *    Laplace   G^(p)(t,s)      = 1/(4 pi) sum_{n<=p} |t-c|^n/|s-c|^{n+1} P_n(cos g)
 *              n_s . grad_s G^(p)   (double layer, Appendix A)
 *              n_t . grad_t G^(p)   (target-normal derivative S', Appendix A)
 *    Helmholtz G_k^(p)(t,s)    = ik/(4 pi) sum_{n<=p} (2n+1) j_n(k|t-c|)
 *                                   h_n(k|s-c|) P_n(cos g)
 *              and its grad_s / grad_t forms (Appendix A).
 *    cos g = (t-c).(s-c)/(|t-c||s-c|); powers by pow(); P_n by Bonnet's
 *    recurrence and P_n' by P'_{n+1} = x P'_n + (n+1) P_n.
 *
 *  Path B -- conventional QBX, Sec. 2.1: local coefficients
 *    L_n^m = sum_s w mu Y_n^{-m}(s-c) / ((2n+1)|s-c|^{n+1})          (eq. local-coeffs)
 *    u(t)  = sum_{n<=p} sum_m L_n^m |t-c|^n Y_n^m(t-c)                 (eq. local-expansion)
 *    with Y_n^m as in eq. sph-harm (no Condon-Shortley phase: it cancels).
 *    Helmholtz replaces 1/((2n+1)|s-c|^{n+1}) |t-c|^n by ik h_n(k|s-c|) j_n(k|t-c|)
 *    (the addition theorem of Appendix A combined with eq. legendre-addition-identity).
 *    Derivatives (double layer, S') are taken with forward-mode dual numbers
 *    (s -> s + eps n_s, t -> t + eps n_t), exact to rounding.
 *
 *  Point kernels -- the un-expanded Green's functions 1/(4 pi r), e^{ikr}/(4 pi r)
 *    and their normal derivatives summed over the same lists (the p -> infinity
 *    limit of path A for convergent pairs, eq. laplace-potential-expansion).
 *
 *  Special functions: j_n by Miller's downward recurrence normalised by
 *  j_0 = sin z/z (or j_1), y_n by upward recurrence from y_0, y_1, h_n = j_n + i y_n
 *  (first kind), derivatives f_n' = f_{n-1} - (n+1)/z f_n, f_0' = -f_1.  Path B
 *  uses the same special-function routines as path A; they are pinned on their
 *  own against closed forms, Wronskians and library routines.
 *
 *  Per-target sums use Neumaier compensated summation.
 *
 * Pins (tests/test_oracle_*.py): path A == path B to rounding (the addition
 * theorem, eq. tsqbx); convergence to the point kernels with the closed-form
 * Laplace tail bound; p = 0, rho = 0 and collinear closed forms; Legendre /
 * Bessel closed forms and library routines; high-precision brute force on tiny
 * cases.  No function here is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_P_MAX 40

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ layout */

/* Geometry and pair lists, mirroring the problem statement of Sec. 3.3/Alg. 1:
 * sources with weights and normals, centers, targets mapped to centers, and per
 * center group a CSR list of half-open source index ranges.  Coordinates are
 * stored SoA: xyz[0..n) = x, xyz[n..2n) = y, xyz[2n..3n) = z. */
typedef struct {
    int64_t n_src;
    const double *src_xyz;     /* [3*n_src] */
    const double *src_weight;  /* [n_src]   */
    const double *src_normal;  /* [3*n_src] or NULL */
    int64_t n_ctr;
    const double *ctr_xyz;     /* [3*n_ctr] */
    int64_t n_tgt;
    const double *tgt_xyz;     /* [3*n_tgt] */
    const int32_t *tgt_center; /* [n_tgt] */
    const double *tgt_normal;  /* [3*n_tgt] or NULL (only for S') */
    int64_t n_group;
    const int32_t *ctr_group;          /* [n_ctr] */
    const int64_t *group_range_start;  /* [n_group+1] */
    const int32_t *range_begin;        /* [nnz] */
    const int32_t *range_end;          /* [nnz] */
} oracle_geom;

/* ------------------------------------------------- compensated summation */

typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else                       a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------- Legendre P_n(x) */

/* P_0..P_p and P'_0..P'_p at x.  Bonnet: (n+1)P_{n+1} = (2n+1)x P_n - n P_{n-1};
 * derivative: P'_{n+1} = x P'_n + (n+1) P_n (valid at x = +-1, no division). */
int oracle_legendre(int p, double x, double *P, double *dP)
{
    if (p < 0 || p > ORACLE_P_MAX) return -1;
    P[0] = 1.0;
    if (dP) dP[0] = 0.0;
    if (p >= 1) { P[1] = x; if (dP) dP[1] = 1.0; }
    for (int n = 1; n < p; ++n) {
        P[n + 1] = ((2.0 * n + 1.0) * x * P[n] - n * P[n - 1]) / (n + 1.0);
        if (dP) dP[n + 1] = x * dP[n] + (n + 1.0) * P[n];
    }
    return 0;
}

/* ---------------------------------------------- spherical Bessel functions */

/* j_0..j_nmax at real z >= 0 by Miller's downward recurrence
 * f_{n-1} = (2n+1)/z f_n - f_{n+1}, started at N = nmax + 20 + ceil(z) with
 * f_{N+1} = 0, f_N = 1e-30 (rescaled when large), renormalised against j_0 = sin z / z or
 * j_1 = sin z / z^2 - cos z / z, whichever is larger in magnitude. */
int oracle_sph_jn(int nmax, double z, double *j)
{
    if (nmax < 0 || nmax > ORACLE_P_MAX + 2 || z < 0.0) return -1;
    if (z == 0.0) {
        j[0] = 1.0;
        for (int n = 1; n <= nmax; ++n) j[n] = 0.0;
        return 0;
    }
    int N = nmax + 20 + (int)ceil(z);
    double *f = (double *)malloc(sizeof(double) * (size_t)(N + 2));
    if (!f) return -2;
    f[N + 1] = 0.0;
    f[N] = 1e-30;
    for (int n = N; n >= 1; --n) {
        f[n - 1] = (2.0 * n + 1.0) / z * f[n] - f[n + 1];
        if (fabs(f[n - 1]) > 1e250) {            /* rescale to avoid overflow */
            for (int m = n - 1; m <= N + 1; ++m) f[m] *= 1e-250;
        }
    }
    double j0 = sin(z) / z;
    double j1 = sin(z) / (z * z) - cos(z) / z;
    double scale = (fabs(j0) >= fabs(j1)) ? j0 / f[0] : j1 / f[1];
    for (int n = 0; n <= nmax; ++n) j[n] = f[n] * scale;
    free(f);
    return 0;
}

/* y_0..y_nmax at real z > 0 by upward recurrence y_{n+1} = (2n+1)/z y_n - y_{n-1}. */
int oracle_sph_yn(int nmax, double z, double *y)
{
    if (nmax < 0 || nmax > ORACLE_P_MAX + 2 || !(z > 0.0)) return -1;
    y[0] = -cos(z) / z;
    if (nmax >= 1) y[1] = -cos(z) / (z * z) - sin(z) / z;
    for (int n = 1; n < nmax; ++n) y[n + 1] = (2.0 * n + 1.0) / z * y[n] - y[n - 1];
    return 0;
}

/* Derivatives f'_n = f_{n-1} - (n+1)/z f_n, f'_0 = -f_1 (needs f up to nmax+1). */
static void sph_deriv(int nmax, double z, const double *f, double *df)
{
    df[0] = -f[1];
    for (int n = 1; n <= nmax; ++n) df[n] = f[n - 1] - (n + 1.0) / z * f[n];
}

int oracle_sph_jn_deriv(int nmax, double z, double *dj)
{
    double j[ORACLE_P_MAX + 4];
    if (nmax < 0 || nmax > ORACLE_P_MAX || !(z > 0.0)) return -1;
    if (oracle_sph_jn(nmax + 1, z, j)) return -1;
    sph_deriv(nmax, z, j, dj);
    return 0;
}

int oracle_sph_yn_deriv(int nmax, double z, double *dy)
{
    double y[ORACLE_P_MAX + 4];
    if (nmax < 0 || nmax > ORACLE_P_MAX || !(z > 0.0)) return -1;
    if (oracle_sph_yn(nmax + 1, z, y)) return -1;
    sph_deriv(nmax, z, y, dy);
    return 0;
}

/* ------------------------------------------------------------ dual numbers */

/* Forward-mode dual numbers a + b eps, eps^2 = 0. */
typedef struct { double v, d; } dual;

static dual D(double v, double d) { dual r = {v, d}; return r; }
static dual dadd(dual a, dual b) { return D(a.v + b.v, a.d + b.d); }
static dual dsub(dual a, dual b) { return D(a.v - b.v, a.d - b.d); }
static dual dmul(dual a, dual b) { return D(a.v * b.v, a.v * b.d + a.d * b.v); }
static dual dscale(dual a, double s) { return D(a.v * s, a.d * s); }
static dual ddiv(dual a, dual b)
{
    return D(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
static dual dsqrt(dual a)
{
    double r = sqrt(a.v);
    return D(r, a.d / (2.0 * r));
}

/* complex dual: (re + i im), each a dual */
typedef struct { dual re, im; } cdual;
static cdual CD(dual re, dual im) { cdual r = {re, im}; return r; }
static cdual cdmul(cdual a, cdual b)
{
    return CD(dsub(dmul(a.re, b.re), dmul(a.im, b.im)),
              dadd(dmul(a.re, b.im), dmul(a.im, b.re)));
}

/* ------------------------------------------------------ spherical harmonics */

/* Y_n^m for a direction given by a (dual) vector v != 0, eq. sph-harm:
 *   Y_n^m = sqrt((2n+1)/(4 pi) (n-|m|)!/(n+|m|)!) P_n^{|m|}(cos theta) e^{i m phi}
 * with cos theta = v_z/|v|, phi = atan2(v_y, v_x).  P_n^{|m|}(x) is written as
 * (1-x^2)^{|m|/2} A_n^{|m|}(x) (no Condon-Shortley phase), so that
 * (sin theta)^{|m|} e^{i m phi} = ((v_x + i sgn(m) v_y)/|v|)^{|m|} and the whole
 * expression is smooth in v (dual-number friendly).  A satisfies
 *   A_m^m = (2m-1)!!, A_{m+1}^m = (2m+1) x A_m^m,
 *   (n-m+1) A_{n+1}^m = (2n+1) x A_n^m - (n+m) A_{n-1}^m.
 * Output index n*n + n + m, for 0 <= n <= p, -n <= m <= n. */
static void sph_harm_dual(int p, dual vx, dual vy, dual vz, cdual *Y)
{
    dual r = dsqrt(dadd(dadd(dmul(vx, vx), dmul(vy, vy)), dmul(vz, vz)));
    dual ux = ddiv(vx, r), uy = ddiv(vy, r), x = ddiv(vz, r);
    /* A[n][m] for m <= n <= p */
    dual A[ORACLE_P_MAX + 1][ORACLE_P_MAX + 1];
    for (int m = 0; m <= p; ++m) {
        double dfact = 1.0;                      /* (2m-1)!! */
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
        A[m][m] = D(dfact, 0.0);
        if (m + 1 <= p) A[m + 1][m] = dscale(x, (2.0 * m + 1.0) * dfact);
        for (int n = m + 1; n < p; ++n) {
            dual t1 = dscale(dmul(x, A[n][m]), 2.0 * n + 1.0);
            dual t2 = dscale(A[n - 1][m], (double)(n + m));
            A[n + 1][m] = dscale(dsub(t1, t2), 1.0 / (n - m + 1.0));
        }
    }
    /* powers of (ux + i uy) */
    cdual pw[ORACLE_P_MAX + 1];
    pw[0] = CD(D(1.0, 0.0), D(0.0, 0.0));
    cdual e1 = CD(ux, uy);
    for (int m = 1; m <= p; ++m) pw[m] = cdmul(pw[m - 1], e1);
    for (int n = 0; n <= p; ++n) {
        for (int m = -n; m <= n; ++m) {
            int am = m < 0 ? -m : m;
            double ratio = 1.0;                   /* (n-|m|)!/(n+|m|)! */
            for (int k = n - am + 1; k <= n + am; ++k) ratio /= k;
            double norm = sqrt((2.0 * n + 1.0) / (4.0 * ORACLE_PI) * ratio);
            dual a = dscale(A[n][am], norm);
            cdual e = pw[am];
            if (m < 0) { e.im = dscale(e.im, -1.0); }
            Y[n * n + n + m] = CD(dmul(a, e.re), dmul(a, e.im));
        }
    }
}

/* Plain-double Y_n^m from the literal angles of eq. sph-harm:
 * theta = acos(z/r), phi = atan2(y, x), P_n^{|m|} by the recurrence above
 * times sin(theta)^{|m|}, e^{i m phi} = cos(m phi) + i sin(m phi). */
int oracle_sph_harm(int p, double vx, double vy, double vz, double *Yre, double *Yim)
{
    if (p < 0 || p > ORACLE_P_MAX) return -1;
    double r = sqrt(vx * vx + vy * vy + vz * vz);
    if (!(r > 0.0)) return -1;
    double theta = acos(vz / r), phi = atan2(vy, vx);
    double x = cos(theta), st = sin(theta);
    double A[ORACLE_P_MAX + 1][ORACLE_P_MAX + 1];
    for (int m = 0; m <= p; ++m) {
        double dfact = 1.0;
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
        A[m][m] = dfact;
        if (m + 1 <= p) A[m + 1][m] = (2.0 * m + 1.0) * x * dfact;
        for (int n = m + 1; n < p; ++n)
            A[n + 1][m] = ((2.0 * n + 1.0) * x * A[n][m] - (n + m) * A[n - 1][m]) / (n - m + 1.0);
    }
    for (int n = 0; n <= p; ++n) {
        for (int m = -n; m <= n; ++m) {
            int am = m < 0 ? -m : m;
            double ratio = 1.0;
            for (int k = n - am + 1; k <= n + am; ++k) ratio /= k;
            double norm = sqrt((2.0 * n + 1.0) / (4.0 * ORACLE_PI) * ratio);
            double mag = norm * A[n][am] * pow(st, am);
            Yre[n * n + n + m] = mag * cos(m * phi);
            Yim[n * n + n + m] = mag * sin(m * phi);
        }
    }
    return 0;
}

/* ------------------------------------------------------------ validation */

static int geom_check(const oracle_geom *g)
{
    if (!g || g->n_src < 0 || g->n_ctr < 0 || g->n_tgt < 0 || g->n_group < 0) return -1;
    for (int64_t t = 0; t < g->n_tgt; ++t) {
        int32_t c = g->tgt_center[t];
        if (c < 0 || c >= g->n_ctr) return -1;
    }
    for (int64_t c = 0; c < g->n_ctr; ++c) {
        int32_t q = g->ctr_group[c];
        if (q < 0 || q >= g->n_group) return -1;
    }
    if (g->group_range_start[0] != 0) return -1;
    for (int64_t q = 0; q < g->n_group; ++q)
        if (g->group_range_start[q + 1] < g->group_range_start[q]) return -1;
    int64_t nnz = g->group_range_start[g->n_group];
    for (int64_t i = 0; i < nnz; ++i) {
        if (g->range_begin[i] < 0 || g->range_end[i] < g->range_begin[i] ||
            g->range_end[i] > g->n_src) return -1;
    }
    return 0;
}

/* Number of (target, source) pairs, counting duplicates. */
int64_t oracle_count_pairs(const oracle_geom *g)
{
    if (geom_check(g)) return -1;
    int64_t total = 0;
    for (int64_t t = 0; t < g->n_tgt; ++t) {
        int32_t q = g->ctr_group[g->tgt_center[t]];
        for (int64_t i = g->group_range_start[q]; i < g->group_range_start[q + 1]; ++i)
            total += g->range_end[i] - g->range_begin[i];
    }
    return total;
}

/* Count pairs with |t-c| >= |s-c| (outside the convergence region of the
 * expansion, Appendix A) and pairs with s == c. */
int oracle_count_divergent(const oracle_geom *g, int64_t *n_div, int64_t *n_zero)
{
    if (geom_check(g)) return -1;
    int64_t nd = 0, nz = 0;
    for (int64_t t = 0; t < g->n_tgt; ++t) {
        int32_t c = g->tgt_center[t];
        int32_t q = g->ctr_group[c];
        double tc[3], rho2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            tc[a] = g->tgt_xyz[a * g->n_tgt + t] - g->ctr_xyz[a * g->n_ctr + c];
            rho2 += tc[a] * tc[a];
        }
        for (int64_t i = g->group_range_start[q]; i < g->group_range_start[q + 1]; ++i)
            for (int32_t s = g->range_begin[i]; s < g->range_end[i]; ++s) {
                double R2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double d = g->src_xyz[a * g->n_src + s] - g->ctr_xyz[a * g->n_ctr + c];
                    R2 += d * d;
                }
                if (R2 == 0.0) ++nz;
                else if (rho2 >= R2) ++nd;
            }
    }
    *n_div = nd;
    *n_zero = nz;
    return 0;
}

/* --------------------------------------------------------- shared helpers */

/* Per-pair geometry: tc = t - c, sc = s - c, rho, R, unit vectors and
 * x = cos(gamma).  When rho == 0 the direction of t - c is undefined; the
 * expansions' limits are obtained with that_ = 0 and x = 0 (every term that
 * would use them carries a vanishing factor |t-c|^n, n >= 1, or P'_0 = 0). */
typedef struct {
    double tc[3], sc[3], rho, R, that_[3], shat[3], x;
} pairgeo;

static void pair_geometry(const oracle_geom *g, int64_t t, int32_t c, int32_t s, pairgeo *pg)
{
    double rho2 = 0.0, R2 = 0.0, dot = 0.0;
    for (int a = 0; a < 3; ++a) {
        pg->tc[a] = g->tgt_xyz[a * g->n_tgt + t] - g->ctr_xyz[a * g->n_ctr + c];
        pg->sc[a] = g->src_xyz[a * g->n_src + s] - g->ctr_xyz[a * g->n_ctr + c];
        rho2 += pg->tc[a] * pg->tc[a];
        R2 += pg->sc[a] * pg->sc[a];
        dot += pg->tc[a] * pg->sc[a];
    }
    pg->rho = sqrt(rho2);
    pg->R = sqrt(R2);
    for (int a = 0; a < 3; ++a) {
        pg->shat[a] = pg->sc[a] / pg->R;
        pg->that_[a] = pg->rho > 0.0 ? pg->tc[a] / pg->rho : 0.0;
    }
    pg->x = pg->rho > 0.0 ? dot / (pg->rho * pg->R) : 0.0;
    if (pg->x > 1.0) pg->x = 1.0;
    if (pg->x < -1.0) pg->x = -1.0;
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void load3(const double *soa, int64_t n, int64_t i, double *v)
{
    v[0] = soa[i]; v[1] = soa[n + i]; v[2] = soa[2 * n + i];
}

/* ================================================================ path A */

/* Laplace target-specific expansion, Appendix A:
 *   G^(p)        = 1/(4pi) sum_{n=0}^p rho^n / R^{n+1} P_n(x)
 *   grad_s G^(p) = 1/(4pi) sum_{n=0}^p rho^n / R^{n+2}
 *                   ( -(n+1) shat P_n(x) + (that - shat x) P'_n(x) )
 *   grad_t G^(p) = 1/(4pi) sum_{n=1}^p rho^{n-1} / R^{n+1}
 *                   ( n that P_n(x) + (shat - that x) P'_n(x) )
 * out_slp[i] = sum_s w mu G^(p), out_dlp[i] = sum_s w mu n_s.grad_s G^(p),
 * out_sp[i]  = sum_s w mu n_t.grad_t G^(p)  for target tgt_subset[i] (or i).
 * Any output pointer may be NULL. */
int oracle_tsqbx_laplace(const oracle_geom *g, int p, const double *density,
                         const int64_t *tgt_subset, int64_t n_subset,
                         double *out_slp, double *out_dlp, double *out_sp)
{
    if (p < 0 || p > ORACLE_P_MAX || geom_check(g)) return -1;
    if (out_dlp && !g->src_normal) return -1;
    if (out_sp && !g->tgt_normal) return -1;
    int64_t nt = tgt_subset ? n_subset : g->n_tgt;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        int64_t t = tgt_subset ? tgt_subset[i] : i;
        if (t < 0 || t >= g->n_tgt) { err = -1; continue; }
        int32_t c = g->tgt_center[t];
        int32_t q = g->ctr_group[c];
        double P[ORACLE_P_MAX + 1], dP[ORACLE_P_MAX + 1], nt_[3] = {0, 0, 0};
        if (out_sp) load3(g->tgt_normal, g->n_tgt, t, nt_);
        nsum us = {0, 0}, ud = {0, 0}, up = {0, 0};
        for (int64_t r = g->group_range_start[q]; r < g->group_range_start[q + 1]; ++r) {
            for (int32_t s = g->range_begin[r]; s < g->range_end[r]; ++s) {
                pairgeo pg;
                pair_geometry(g, t, c, s, &pg);
                oracle_legendre(p, pg.x, P, dP);
                double wmu = g->src_weight[s] * density[s];
                if (out_slp) {
                    nsum acc = {0, 0};
                    for (int n = 0; n <= p; ++n)
                        nsum_add(&acc, pow(pg.rho, n) / pow(pg.R, n + 1) * P[n]);
                    nsum_add(&us, wmu * nsum_get(&acc) / (4.0 * ORACLE_PI));
                }
                if (out_dlp) {
                    double ns[3];
                    load3(g->src_normal, g->n_src, s, ns);
                    double shn = dot3(pg.shat, ns), thn = dot3(pg.that_, ns);
                    nsum acc = {0, 0};
                    for (int n = 0; n <= p; ++n) {
                        double f = pow(pg.rho, n) / pow(pg.R, n + 2);
                        double v = -(n + 1.0) * shn * P[n] + (thn - shn * pg.x) * dP[n];
                        nsum_add(&acc, f * v);
                    }
                    nsum_add(&ud, wmu * nsum_get(&acc) / (4.0 * ORACLE_PI));
                }
                if (out_sp) {
                    double thn = dot3(pg.that_, nt_), shn = dot3(pg.shat, nt_);
                    nsum acc = {0, 0};
                    for (int n = 1; n <= p; ++n) {
                        double f = pow(pg.rho, n - 1) / pow(pg.R, n + 1);
                        double v = n * thn * P[n] + (shn - thn * pg.x) * dP[n];
                        nsum_add(&acc, f * v);
                    }
                    nsum_add(&up, wmu * nsum_get(&acc) / (4.0 * ORACLE_PI));
                }
            }
        }
        if (out_slp) out_slp[i] = nsum_get(&us);
        if (out_dlp) out_dlp[i] = nsum_get(&ud);
        if (out_sp) out_sp[i] = nsum_get(&up);
    }
    return err;
}

/* Helmholtz target-specific expansion, Appendix A (h_n = h_n^(1)):
 *   G_k^(p)        = ik/(4pi) sum_{n<=p} (2n+1) j_n(k rho) h_n(kR) P_n(x)
 *   grad_s G_k^(p) = ik/(4pi) sum_{n<=p} (2n+1) j_n(k rho)/R
 *                     ( k (s-c) h'_n(kR) P_n(x) + (that - shat x) h_n(kR) P'_n(x) )
 *   grad_t G_k^(p) = ik/(4pi) sum_{n<=p} (2n+1) h_n(kR)/rho
 *                     ( k (t-c) j'_n(k rho) P_n(x) + (shat - that x) j_n(k rho) P'_n(x) )
 * density and outputs are complex, interleaved (re, im).  At rho == 0 the
 * grad_t form is its limit ik/(4pi) k h_1(kR) shat (only n = 1 survives). */
int oracle_tsqbx_helmholtz(const oracle_geom *g, int p, double k, const double *density,
                           const int64_t *tgt_subset, int64_t n_subset,
                           double *out_slp, double *out_dlp, double *out_sp)
{
    if (p < 0 || p > ORACLE_P_MAX || !(k > 0.0) || geom_check(g)) return -1;
    if (out_dlp && !g->src_normal) return -1;
    if (out_sp && !g->tgt_normal) return -1;
    int64_t nt = tgt_subset ? n_subset : g->n_tgt;
    int err = 0;
    const double complex pref = I * k / (4.0 * ORACLE_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        int64_t t = tgt_subset ? tgt_subset[i] : i;
        if (t < 0 || t >= g->n_tgt) { err = -1; continue; }
        int32_t c = g->tgt_center[t];
        int32_t q = g->ctr_group[c];
        double P[ORACLE_P_MAX + 1], dP[ORACLE_P_MAX + 1];
        double jt[ORACLE_P_MAX + 3], djt[ORACLE_P_MAX + 2];
        double js[ORACLE_P_MAX + 3], ys[ORACLE_P_MAX + 3], djs[ORACLE_P_MAX + 2], dys[ORACLE_P_MAX + 2];
        double nt_[3] = {0, 0, 0};
        if (out_sp) load3(g->tgt_normal, g->n_tgt, t, nt_);
        double rho = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d = g->tgt_xyz[a * g->n_tgt + t] - g->ctr_xyz[a * g->n_ctr + c];
            rho += d * d;
        }
        rho = sqrt(rho);
        oracle_sph_jn(p + 1, k * rho, jt);
        if (rho > 0.0) sph_deriv(p, k * rho, jt, djt);
        nsum us[2] = {{0, 0}, {0, 0}}, ud[2] = {{0, 0}, {0, 0}}, up[2] = {{0, 0}, {0, 0}};
        for (int64_t r = g->group_range_start[q]; r < g->group_range_start[q + 1]; ++r) {
            for (int32_t s = g->range_begin[r]; s < g->range_end[r]; ++s) {
                pairgeo pg;
                pair_geometry(g, t, c, s, &pg);
                oracle_legendre(p, pg.x, P, dP);
                double z = k * pg.R;
                oracle_sph_jn(p + 1, z, js);
                oracle_sph_yn(p + 1, z, ys);
                sph_deriv(p, z, js, djs);
                sph_deriv(p, z, ys, dys);
                double complex wmu = g->src_weight[s] * (density[2 * s] + I * density[2 * s + 1]);
                double complex val;
                if (out_slp) {
                    double complex acc = 0.0;
                    for (int n = 0; n <= p; ++n)
                        acc += (2.0 * n + 1.0) * jt[n] * (js[n] + I * ys[n]) * P[n];
                    val = pref * acc * wmu;
                    nsum_add(&us[0], creal(val)); nsum_add(&us[1], cimag(val));
                }
                if (out_dlp) {
                    double ns[3];
                    load3(g->src_normal, g->n_src, s, ns);
                    double scn = dot3(pg.sc, ns);
                    double tsn = dot3(pg.that_, ns) - dot3(pg.shat, ns) * pg.x;
                    double complex acc = 0.0;
                    for (int n = 0; n <= p; ++n) {
                        double complex h = js[n] + I * ys[n], dh = djs[n] + I * dys[n];
                        acc += (2.0 * n + 1.0) * jt[n] / pg.R *
                               (k * scn * dh * P[n] + tsn * h * dP[n]);
                    }
                    val = pref * acc * wmu;
                    nsum_add(&ud[0], creal(val)); nsum_add(&ud[1], cimag(val));
                }
                if (out_sp) {
                    double complex acc = 0.0;
                    if (rho > 0.0) {
                        double tcn = dot3(pg.tc, nt_);
                        double stn = dot3(pg.shat, nt_) - dot3(pg.that_, nt_) * pg.x;
                        for (int n = 0; n <= p; ++n) {
                            double complex h = js[n] + I * ys[n];
                            acc += (2.0 * n + 1.0) * h / rho *
                                   (k * tcn * djt[n] * P[n] + stn * jt[n] * dP[n]);
                        }
                    } else if (p >= 1) {
                        acc = k * (js[1] + I * ys[1]) * dot3(pg.shat, nt_);
                    }
                    val = pref * acc * wmu;
                    nsum_add(&up[0], creal(val)); nsum_add(&up[1], cimag(val));
                }
            }
        }
        if (out_slp) { out_slp[2 * i] = nsum_get(&us[0]); out_slp[2 * i + 1] = nsum_get(&us[1]); }
        if (out_dlp) { out_dlp[2 * i] = nsum_get(&ud[0]); out_dlp[2 * i + 1] = nsum_get(&ud[1]); }
        if (out_sp) { out_sp[2 * i] = nsum_get(&up[0]); out_sp[2 * i + 1] = nsum_get(&up[1]); }
    }
    return err;
}

/* ================================================================ path B */

static cdual cd_from(double complex z) { return CD(D(creal(z), 0.0), D(cimag(z), 0.0)); }
static cdual cdadd(cdual a, cdual b) { return CD(dadd(a.re, b.re), dadd(a.im, b.im)); }
static cdual cd_real(dual a) { return CD(a, D(0.0, 0.0)); }

/* Conventional QBX through spherical-harmonic local coefficients (Sec. 2.1,
 * eqs. local-coeffs and local-expansion; Helmholtz through the addition
 * theorem of Appendix A with eq. legendre-addition-identity).  For the target
 * tgt_subset[i] the coefficients of its center are formed from every source of
 * the center's group lists, then evaluated at the target.
 *   kernel 0 (Laplace):   radial factors 1/((2n+1) R^{n+1}) and rho^n
 *   kernel 1 (Helmholtz): radial factors ik h_n(kR) and j_n(k rho)
 * The double layer is the eps-part of the coefficients for s -> s + eps n_s,
 * S' the eps-part of the evaluation for t -> t + eps n_t.  Outputs are
 * complex interleaved for Helmholtz, real for Laplace. */
static int qbx_conventional(const oracle_geom *g, int kernel, int p, double k,
                            const double *density, const int64_t *tgt_subset, int64_t n_subset,
                            double *out_slp, double *out_dlp, double *out_sp)
{
    if (p < 0 || p > ORACLE_P_MAX || geom_check(g)) return -1;
    if (kernel == 1 && !(k > 0.0)) return -1;
    if (out_dlp && !g->src_normal) return -1;
    if (out_sp && !g->tgt_normal) return -1;
    int64_t nt = tgt_subset ? n_subset : g->n_tgt;
    int ncoef = (p + 1) * (p + 1);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < nt; ++i) {
        int64_t t = tgt_subset ? tgt_subset[i] : i;
        if (t < 0 || t >= g->n_tgt) { err = -1; continue; }
        int32_t c = g->tgt_center[t];
        int32_t q = g->ctr_group[c];
        cdual *L = (cdual *)calloc((size_t)ncoef, sizeof(cdual));
        cdual *Y = (cdual *)malloc(sizeof(cdual) * (size_t)ncoef);
        if (!L || !Y) { free(L); free(Y); err = -2; continue; }
        double cx[3];
        load3(g->ctr_xyz, g->n_ctr, c, cx);
        /* ---- coefficient formation */
        for (int64_t r = g->group_range_start[q]; r < g->group_range_start[q + 1]; ++r) {
            for (int32_t s = g->range_begin[r]; s < g->range_end[r]; ++s) {
                double sx[3], ns[3] = {0, 0, 0};
                load3(g->src_xyz, g->n_src, s, sx);
                if (out_dlp) load3(g->src_normal, g->n_src, s, ns);
                dual v[3];
                for (int a = 0; a < 3; ++a) v[a] = D(sx[a] - cx[a], ns[a]);
                dual R = dsqrt(dadd(dadd(dmul(v[0], v[0]), dmul(v[1], v[1])), dmul(v[2], v[2])));
                sph_harm_dual(p, v[0], v[1], v[2], Y);
                double complex wmu = kernel == 0
                    ? g->src_weight[s] * density[s]
                    : g->src_weight[s] * (density[2 * s] + I * density[2 * s + 1]);
                double hj[ORACLE_P_MAX + 3], hy[ORACLE_P_MAX + 3], dhj[ORACLE_P_MAX + 2], dhy[ORACLE_P_MAX + 2];
                if (kernel == 1) {
                    oracle_sph_jn(p + 1, k * R.v, hj);
                    oracle_sph_yn(p + 1, k * R.v, hy);
                    sph_deriv(p, k * R.v, hj, dhj);
                    sph_deriv(p, k * R.v, hy, dhy);
                }
                dual Rpow = R;                           /* R^{n+1} */
                for (int n = 0; n <= p; ++n) {
                    cdual radial;
                    if (kernel == 0) {
                        radial = cd_real(ddiv(D(1.0, 0.0), dscale(Rpow, 2.0 * n + 1.0)));
                        Rpow = dmul(Rpow, R);
                    } else {
                        /* ik h_n(k R) with R dual: h_n + eps k R' h'_n */
                        double complex h = hj[n] + I * hy[n], dh = dhj[n] + I * dhy[n];
                        double complex a = I * k * h, b = I * k * (k * R.d) * dh;
                        radial = CD(D(creal(a), creal(b)), D(cimag(a), cimag(b)));
                    }
                    cdual f = cdmul(cd_from(wmu), radial);
                    for (int m = -n; m <= n; ++m)
                        L[n * n + n + m] = cdadd(L[n * n + n + m], cdmul(f, Y[n * n + n - m]));
                }
            }
        }
        /* ---- evaluation at the target */
        double tx[3], ntv[3] = {0, 0, 0};
        load3(g->tgt_xyz, g->n_tgt, t, tx);
        if (out_sp) load3(g->tgt_normal, g->n_tgt, t, ntv);
        dual v[3];
        for (int a = 0; a < 3; ++a) v[a] = D(tx[a] - cx[a], ntv[a]);
        dual rho = dsqrt(dadd(dadd(dmul(v[0], v[0]), dmul(v[1], v[1])), dmul(v[2], v[2])));
        int nmax = p;
        if (rho.v == 0.0) {            /* value: only n = 0 survives, its Y constant (S': below) */
            nmax = 0;
            v[0] = D(0.0, 0.0); v[1] = D(0.0, 0.0); v[2] = D(1.0, 0.0);
            rho = D(0.0, 0.0);
        }
        sph_harm_dual(p, v[0], v[1], v[2], Y);
        double tj[ORACLE_P_MAX + 3], tdj[ORACLE_P_MAX + 2];
        if (kernel == 1) {
            oracle_sph_jn(p + 1, k * rho.v, tj);
            if (rho.v > 0.0) sph_deriv(p, k * rho.v, tj, tdj);
        }
        nsum acc[3][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
        dual rpow = D(1.0, 0.0);                 /* rho^n */
        for (int n = 0; n <= nmax; ++n) {
            dual radial;
            if (kernel == 0) { radial = rpow; rpow = dmul(rpow, rho); }
            else radial = D(tj[n], rho.v > 0.0 ? k * rho.d * tdj[n] : 0.0);
            for (int m = -n; m <= n; ++m) {
                cdual e = cdmul(cd_real(radial), Y[n * n + n + m]);
                cdual Lc = L[n * n + n + m];
                /* value:  L.v * e.v ; dlp: L.d * e.v ; sp: L.v * e.d */
                double complex Lv = Lc.re.v + I * Lc.im.v, Ld = Lc.re.d + I * Lc.im.d;
                double complex ev = e.re.v + I * e.im.v, ed = e.re.d + I * e.im.d;
                double complex a0 = Lv * ev, a1 = Ld * ev, a2 = Lv * ed;
                nsum_add(&acc[0][0], creal(a0)); nsum_add(&acc[0][1], cimag(a0));
                nsum_add(&acc[1][0], creal(a1)); nsum_add(&acc[1][1], cimag(a1));
                nsum_add(&acc[2][0], creal(a2)); nsum_add(&acc[2][1], cimag(a2));
            }
        }
        if (out_sp && rho.v == 0.0 && p >= 1) {
            /* S' at t = c: the limit along n_t.  Only n = 1 has a radial
             * factor with a nonzero slope at rho = 0 (rho for Laplace, j_1(k rho)
             * ~ k rho / 3 for Helmholtz), and its angular factor is constant
             * along the ray, so the derivative is slope * Y_1^m(n_t). */
            const double slope = kernel == 0 ? 1.0 : k / 3.0;
            sph_harm_dual(p, D(ntv[0], 0.0), D(ntv[1], 0.0), D(ntv[2], 0.0), Y);
            for (int m = -1; m <= 1; ++m) {
                cdual Lc = L[1 + 1 + m];
                double complex Lv = Lc.re.v + I * Lc.im.v;
                double complex yv = Y[1 + 1 + m].re.v + I * Y[1 + 1 + m].im.v;
                double complex a2 = Lv * slope * yv;
                nsum_add(&acc[2][0], creal(a2)); nsum_add(&acc[2][1], cimag(a2));
            }
        }
        double *outs[3] = {out_slp, out_dlp, out_sp};
        for (int o = 0; o < 3; ++o) {
            if (!outs[o]) continue;
            if (kernel == 0) outs[o][i] = nsum_get(&acc[o][0]);
            else { outs[o][2 * i] = nsum_get(&acc[o][0]); outs[o][2 * i + 1] = nsum_get(&acc[o][1]); }
        }
        free(L);
        free(Y);
    }
    return err;
}

int oracle_qbx_laplace(const oracle_geom *g, int p, const double *density,
                       const int64_t *tgt_subset, int64_t n_subset,
                       double *out_slp, double *out_dlp, double *out_sp)
{
    return qbx_conventional(g, 0, p, 0.0, density, tgt_subset, n_subset, out_slp, out_dlp, out_sp);
}

int oracle_qbx_helmholtz(const oracle_geom *g, int p, double k, const double *density,
                         const int64_t *tgt_subset, int64_t n_subset,
                         double *out_slp, double *out_dlp, double *out_sp)
{
    return qbx_conventional(g, 1, p, k, density, tgt_subset, n_subset, out_slp, out_dlp, out_sp);
}

/* ========================================================= point kernels */

/* Un-expanded kernels over the same lists:
 *   Laplace   G = 1/(4 pi r), n_s.grad_s G = n_s.(t-s)/(4 pi r^3), n_t.grad_t G = -n_t.(t-s)/(4 pi r^3)
 *   Helmholtz G = e^{ikr}/(4 pi r), grad_s G = e^{ikr}(1 - ikr)(t-s)/(4 pi r^3) = -grad_t G
 * kernel 0 = Laplace (real density/outputs), 1 = Helmholtz (complex interleaved). */
int oracle_point_potential(const oracle_geom *g, int kernel, double k, const double *density,
                           const int64_t *tgt_subset, int64_t n_subset,
                           double *out_slp, double *out_dlp, double *out_sp)
{
    if (geom_check(g)) return -1;
    if (out_dlp && !g->src_normal) return -1;
    if (out_sp && !g->tgt_normal) return -1;
    int64_t nt = tgt_subset ? n_subset : g->n_tgt;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; ++i) {
        int64_t t = tgt_subset ? tgt_subset[i] : i;
        if (t < 0 || t >= g->n_tgt) { err = -1; continue; }
        int32_t q = g->ctr_group[g->tgt_center[t]];
        double tx[3], ntv[3] = {0, 0, 0};
        load3(g->tgt_xyz, g->n_tgt, t, tx);
        if (out_sp) load3(g->tgt_normal, g->n_tgt, t, ntv);
        nsum acc[3][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
        for (int64_t r = g->group_range_start[q]; r < g->group_range_start[q + 1]; ++r) {
            for (int32_t s = g->range_begin[r]; s < g->range_end[r]; ++s) {
                double sx[3], ns[3] = {0, 0, 0}, ts[3];
                load3(g->src_xyz, g->n_src, s, sx);
                if (out_dlp) load3(g->src_normal, g->n_src, s, ns);
                for (int a = 0; a < 3; ++a) ts[a] = tx[a] - sx[a];
                double r2 = dot3(ts, ts), rr = sqrt(r2);
                double complex wmu = kernel == 0
                    ? g->src_weight[s] * density[s]
                    : g->src_weight[s] * (density[2 * s] + I * density[2 * s + 1]);
                double complex G, dG;                /* G and (dG/dr)/r  */
                if (kernel == 0) {
                    G = 1.0 / (4.0 * ORACLE_PI * rr);
                    dG = 1.0 / (4.0 * ORACLE_PI * rr * r2);          /* grad_s G = dG (t-s) */
                } else {
                    double complex e = cexp(I * k * rr);
                    G = e / (4.0 * ORACLE_PI * rr);
                    dG = e * (1.0 - I * k * rr) / (4.0 * ORACLE_PI * rr * r2);
                }
                double complex v[3] = {wmu * G, wmu * dG * dot3(ns, ts), -wmu * dG * dot3(ntv, ts)};
                for (int o = 0; o < 3; ++o) {
                    nsum_add(&acc[o][0], creal(v[o]));
                    nsum_add(&acc[o][1], cimag(v[o]));
                }
            }
        }
        double *outs[3] = {out_slp, out_dlp, out_sp};
        for (int o = 0; o < 3; ++o) {
            if (!outs[o]) continue;
            if (kernel == 0) outs[o][i] = nsum_get(&acc[o][0]);
            else { outs[o][2 * i] = nsum_get(&acc[o][0]); outs[o][2 * i + 1] = nsum_get(&acc[o][1]); }
        }
    }
    return err;
}
