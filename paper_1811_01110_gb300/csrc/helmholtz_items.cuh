// helmholtz_items.cuh -- the Helmholtz TSQBX kernel (arithmetic described in
// helmholtz.cu) and its dispatch over p.  helmholtz.cu instantiates the
// single/double-layer variants, helmholtz_sp.cu the ones that also form S'.
#pragma once

#include <utility>

#include "internal.cuh"

namespace tsqbx {
namespace {

// Rows of the warp's staging tile: x, y, z, Re and Im of w mu (of each of the
// nrhs densities), and for the double layer the normal's three components;
// each row holds DevGeom::tile sources.
__host__ __device__ constexpr int helmholtz_tile_rows(bool dlp, int nrhs = 1)
{
    return dlp ? 8 : 3 + 2 * nrhs;
}

// Per-target radial factors, orders 0..P (z = k rho):
//   cj[n]  = (2n+1) kappa_n j_n(z)
//   caj[n] = (2n+1) kappa_n k j_n'(z) (that.n_t)        (S' only)
// j_n by Miller's downward recurrence (f_{n-1} = (2n+1)/z f_n - f_{n+1}),
// started P + 20 + ceil(z) orders up and normalised against j_0 = sin z / z
// or j_1 = sin z / z^2 - cos z / z, whichever is larger; j_n' = (n/z) j_n -
// j_{n+1} (the run also yields j_{P+1}).  z = 0: j_0 = 1, j_1' = 1/3, rest 0.
// The run above P keeps two scalars; orders P+1..0 are unrolled, so every
// array here stays in registers.
template <int P, bool SP>
__device__ __forceinline__ void helmholtz_target_factors(double k, double rho, double tdot, double (&cj)[P + 1],
                                                         double (&caj)[SP ? P + 1 : 1])
{
    const double z = k * rho;
    double jn[P + 2];
    if (z == 0.0) {
#pragma unroll
        for (int n = 0; n <= P + 1; ++n) jn[n] = n == 0 ? 1.0 : 0.0;
    } else {
        const double zinv = 1.0 / z;
        const int N = P + 20 + (int)fmin(ceil(z), 1.0e6);   // no int overflow for huge k rho
        double fa = 0.0, fb = 1e-30;           // f_{n+1}, f_n
        for (int n = N; n > P; --n) {
            const double fnew = (2.0 * n + 1.0) * zinv * fb - fa;
            fa = fb;
            fb = fnew;
            if (fabs(fb) > 1e200) { fa *= 1e-200; fb *= 1e-200; }
        }
        jn[P + 1] = fa;
        jn[P] = fb;
#pragma unroll
        for (int n = P; n >= 1; --n) {
            jn[n - 1] = (2.0 * n + 1.0) * zinv * jn[n] - jn[n + 1];
            if (fabs(jn[n - 1]) > 1e200) {
#pragma unroll
                for (int m = n - 1; m <= P + 1; ++m) jn[m] *= 1e-200;
            }
        }
        double sn, cs;
        sincos(z, &sn, &cs);
        const double j0 = sn * zinv;
        const double j1 = (sn * zinv - cs) * zinv;
        const double scale = fabs(j1) > fabs(j0) ? j1 / jn[1] : j0 / jn[0];
#pragma unroll
        for (int n = 0; n <= P + 1; ++n) jn[n] *= scale;
    }
    double kap = 1.0;                                   // kappa_n
    const double zinv = z == 0.0 ? 0.0 : 1.0 / z;
#pragma unroll
    for (int n = 0; n <= P; ++n) {
        const double f = (2.0 * n + 1.0) * kap;
        cj[n] = f * jn[n];
        if (SP) {
            const double jd = z == 0.0 ? (n == 1 ? 1.0 / 3.0 : 0.0) : fma(n * zinv, jn[n], -jn[n + 1]);
            caj[SP ? n : 0] = f * k * jd * tdot;
        }
        kap *= (2.0 * n + 1.0) / (n + 1.0);
    }
}

// Complex helpers on (re, im) pairs.
__device__ __forceinline__ void cfma(double c, double gr, double gi, double &ar, double &ai)
{
    ar = fma(c, gr, ar);
    ai = fma(c, gi, ai);
}

// NRHS > 1 (single layer only): the densities ev.n_rhs = NRHS share every
// per-pair quantity -- geometry, recurrences, e^{ikR} and the Clenshaw sum --
// and differ only in the final weight, applied with the same operations as
// for one density, so each result is bit-identical to its own evaluation.
template <int P, bool DLP, bool SP, int NRHS = 1>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
helmholtz_kernel(const DevGeom g, const DevEval ev)
{
    static_assert(NRHS == 1 || (!DLP && !SP), "several densities: single layer only");
    constexpr int kRows = helmholtz_tile_rows(DLP, NRHS);
    extern __shared__ __align__(16) double smem_helm[];
    const int tile = g.tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    const Item it = g.items[item];
    const int L = it.L;
    const int j = lane / L, sub = lane - j * L;
    const bool active = j < it.n_tgt;
    const double k = ev.k, kinv = 1.0 / ev.k;
    double cx = 0, cy = 0, cz = 0, ex = 0, ey = 0, ez = 0, rhoinv = 0;
    double tx = 0, ty = 0, tz = 0, tdot = 0, b1 = 0;   // n_t, that.n_t, rho = 0 limit of k j_1/rho
    double cj[P + 1];
    double caj[SP ? P + 1 : 1];
#pragma unroll
    for (int n = 0; n <= P; ++n) cj[n] = 0.0;
#pragma unroll
    for (int n = 0; n < (SP ? P + 1 : 1); ++n) caj[n] = 0.0;
    if (active) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double4_32a e = g.slot_e[it.slot_begin + j];
        cx = c.x; cy = c.y; cz = c.z;
        ex = e.x; ey = e.y; ez = e.z;
        const double rho = sqrt(e.w);
        rhoinv = rho > 0.0 ? 1.0 / rho : 0.0;
        if (SP) {
            const double4_32a tn = g.slot_n[it.slot_begin + j];
            tx = tn.x; ty = tn.y; tz = tn.z;
            tdot = fma(ex, tx, fma(ey, ty, ez * tz)) * rhoinv;
            b1 = (rho > 0.0 || P < 1) ? 0.0 : k;
        }
        helmholtz_target_factors<P, SP>(k, rho, tdot, cj, caj);
    }
    ListWalk walk(g, g.item_walk[item]);
    const int src_hi = it.src_hi;
    double *const Tbase = smem_helm + (size_t)warp * kRows * tile;
    auto T = [&](int row) { return Tbase + row * tile; };
    double acc_re = 0.0, acc_im = 0.0, dacc_re = 0.0, dacc_im = 0.0, pacc_re = 0.0, pacc_im = 0.0;
    double xacc_re[NRHS > 1 ? NRHS - 1 : 1], xacc_im[NRHS > 1 ? NRHS - 1 : 1];   // densities 1..NRHS-1
#pragma unroll
    for (int r = 0; r < (NRHS > 1 ? NRHS - 1 : 1); ++r) xacc_re[r] = xacc_im[r] = 0.0;

    for (int base = it.src_lo; base < src_hi; base += tile) {
        const int cnt = min(tile, src_hi - base);
        for (int kk = lane; kk < cnt; kk += 32) {
            int s = walk.at(base + kk);
            double2 wm = make_double2(0.0, 0.0);
            const bool in_range = (unsigned)s < (unsigned)g.n_src;
            if (!in_range) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu_c[s];
            const double4_32a pw = g.src_pw[s];
            T(0)[kk] = pw.x; T(1)[kk] = pw.y; T(2)[kk] = pw.z;
            T(3)[kk] = wm.x; T(4)[kk] = wm.y;
#pragma unroll
            for (int r = 1; r < NRHS; ++r) {
                const double2 wr = in_range ? ev.wmu_c[r * ev.rhs_src_stride + s] : make_double2(0.0, 0.0);
                T(3 + 2 * r)[kk] = wr.x; T(4 + 2 * r)[kk] = wr.y;
            }
            if (DLP) {
                const double4_32a n = g.src_n[s];
                T(kRows - 3)[kk] = n.x; T(kRows - 2)[kk] = n.y; T(kRows - 1)[kk] = n.z;
            }
        }
        __syncwarp();
        if (active) {
            for (int kk = sub; kk < cnt; kk += L) {
                const double dx = T(0)[kk] - cx, dy = T(1)[kk] - cy, dz = T(2)[kk] - cz;
                const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const double rinv = rsqrt(R2);
                const double x = fma(dx, ex, fma(dy, ey, dz * ez)) * rinv * rhoinv;
                const double w = rinv * kinv;               // 1/z
                const double z = k * (R2 * rinv);
                // Every layer is a sum over n of g_n (h_n = e^{iz} g_n) with real
                // coefficients c_n.  The g_n obey g_{n+1} = (2n+1) w g_n - g_{n-1}
                // (g_{-1} = w, g_0 = -i w, g_1 = -w - i w^2), so each sum goes by
                // Clenshaw's backward recurrence b_n = c_n + (2n+1) w b_{n+1} -
                // b_{n+2}: sum = (c_0 - b_2) g_0 + b_1 g_1, in real arithmetic.
                //  * single layer: c_n = a_n = cj_n T_n;
                //  * double layer, kah D1 + u D2 with D1 = sum a_n h_n'/e^{iz} and
                //    h_n' = e^{iz} (g_{n-1} - (n+1) w g_n):  D1 = a_0 w + sum e_n g_n,
                //    e_n = a_{n+1} - (n+1) w a_n (a_{P+1} = 0);  c_n = kah e_n +
                //    u cj_n T'_n, and kah a_0 w adds to the real part;
                //  * S', C B + Pa:  c_n = (C/rho) cj_n T'_n + caj_n T_n, plus C b1 on
                //    g_1 (the rho = 0 limit of the n = 1 term).
                // T_n and T'_n go forward first and stay in registers.
                double kah = 0.0, u = 0.0, Cr = 0.0, Cl = 0.0;
                if (DLP) {
                    // n_s.grad_s: R' = a/R, x' = (1/R) ((e.n_s)/rho - (a/R) x), a = d.n_s
                    const double nx = T(kRows - 3)[kk], ny = T(kRows - 2)[kk], nz = T(kRows - 1)[kk];
                    const double ah = fma(dx, nx, fma(dy, ny, dz * nz)) * rinv;
                    u = (fma(ex, nx, fma(ey, ny, ez * nz)) * rhoinv - ah * x) * rinv;
                    kah = k * ah;
                }
                if (SP) {
                    // n_t.grad_t: rho' = that.n_t, x' = (1/rho) ((d.n_t)/R - (that.n_t) x)
                    const double C = fma(dx, tx, fma(dy, ty, dz * tz)) * rinv - tdot * x;
                    Cr = C * rhoinv;
                    Cl = C * b1;
                }
                double Tv[P + 1], Uv[(DLP || SP) ? P + 1 : 1];
                Tv[0] = 1.0;
                if (P >= 1) Tv[1] = x;
                if (DLP || SP) {
                    Uv[0] = 0.0;
                    if (P >= 1) Uv[(DLP || SP) ? 1 : 0] = 1.0;
                }
#pragma unroll
                for (int n = 1; n < P; ++n) {
                    Tv[n + 1] = fma(x, Tv[n], -rec_beta(n) * Tv[n - 1]);
                    if (DLP || SP) Uv[n + 1] = fma(-rec_beta(n), Uv[n - 1], fma(x, Uv[n], Tv[n]));
                }
                double bA1 = 0.0, bA2 = 0.0, bD1 = 0.0, bD2 = 0.0, bS1 = 0.0, bS2 = 0.0, a_next = 0.0;
                if constexpr (P >= 1) {
                    // n = P: b_{P+1} = b_{P+2} = 0, so b_P = c_P (a product by a
                    // zero b would still cost an operation: IEEE x * 0 is not 0
                    // for every x)
                    constexpr int n = P;
                    if (DLP) {
                        const double an = cj[n] * Tv[n];
                        bA1 = an;
                        bD1 = fma(kah, (-(n + 1.0) * w) * an, u * (cj[n] * Uv[n]));
                        a_next = an;
                    } else {
                        bA1 = cj[n] * Tv[n];
                    }
                    if (SP) {
                        double hn = fma(Cr, cj[n] * Uv[(DLP || SP) ? n : 0], caj[SP ? n : 0] * Tv[n]);
                        if (n == 1) hn += Cl;
                        bS1 = hn;
                    }
                }
#pragma unroll
                for (int n = P - 1; n >= 1; --n) {
                    const double t = (2.0 * n + 1.0) * w;
                    if (DLP) {
                        const double an = cj[n] * Tv[n];
                        const double bA = fma(t, bA1, an - bA2);
                        bA2 = bA1; bA1 = bA;
                        const double en = fma(-(n + 1.0) * w, an, a_next);
                        const double bD = fma(t, bD1, fma(kah, en, u * (cj[n] * Uv[n])) - bD2);
                        bD2 = bD1; bD1 = bD;
                        a_next = an;
                    } else {
                        const double bA = fma(t, bA1, fma(cj[n], Tv[n], -bA2));
                        bA2 = bA1; bA1 = bA;
                    }
                    if (SP) {
                        double hn = fma(Cr, cj[n] * Uv[(DLP || SP) ? n : 0], caj[SP ? n : 0] * Tv[n]);
                        if (n == 1) hn += Cl;
                        const double bS = fma(t, bS1, hn - bS2);
                        bS2 = bS1; bS1 = bS;
                    }
                }
                // (c_0 - b_2) g_0 + b_1 g_1 = (-w b_1, -w (c_0 - b_2 + w b_1))
                auto close = [&](double c0, double bb1, double bb2, double &re, double &im) {
                    re = -w * bb1;
                    im = -w * fma(w, bb1, c0 - bb2);
                };
                double Ar, Ai;
                close(cj[0], bA1, bA2, Ar, Ai);
                double sn, cs;
                sincos(z, &sn, &cs);
                const double wr = T(3)[kk], wi = T(4)[kk];
                // out += ik e^{iz} (X) (w mu):  with v = e^{iz} X, ik v = (-k v_i, k v_r)
                auto accumulate = [&](double Xr, double Xi, double &or_, double &oi) {
                    const double vr = fma(cs, Xr, -sn * Xi), vi = fma(sn, Xr, cs * Xi);
                    const double ur = -k * vi, ui = k * vr;
                    or_ = fma(ur, wr, fma(-ui, wi, or_));
                    oi = fma(ur, wi, fma(ui, wr, oi));
                };
                accumulate(Ar, Ai, acc_re, acc_im);
                if constexpr (NRHS > 1) {
                    // the other densities: the same operations with their own weights
                    const double vr = fma(cs, Ar, -sn * Ai), vi = fma(sn, Ar, cs * Ai);
                    const double ur = -k * vi, ui = k * vr;
#pragma unroll
                    for (int r = 1; r < NRHS; ++r) {
                        const double w2r = T(3 + 2 * r)[kk], w2i = T(4 + 2 * r)[kk];
                        xacc_re[r - 1] = fma(ur, w2r, fma(-ui, w2i, xacc_re[r - 1]));
                        xacc_im[r - 1] = fma(ur, w2i, fma(ui, w2r, xacc_im[r - 1]));
                    }
                }
                if (DLP) {
                    double Dr, Di;
                    close(kah * fma(-w, cj[0], a_next), bD1, bD2, Dr, Di);     // a_next = a_1 (0 if P = 0)
                    accumulate(fma(kah * cj[0], w, Dr), Di, dacc_re, dacc_im);
                }
                if (SP) {
                    double Sr, Si;
                    close(caj[0], bS1, bS2, Sr, Si);                           // c_0 = caj_0 (T'_0 = 0)
                    accumulate(Sr, Si, pacc_re, pacc_im);
                }
            }
        }
        __syncwarp();
    }
    for (int off = 1; off < L; off <<= 1) {
        const double vr = __shfl_down_sync(0xffffffffu, acc_re, off);
        const double vi = __shfl_down_sync(0xffffffffu, acc_im, off);
        const double dr = DLP ? __shfl_down_sync(0xffffffffu, dacc_re, off) : 0.0;
        const double di = DLP ? __shfl_down_sync(0xffffffffu, dacc_im, off) : 0.0;
        const double pr = SP ? __shfl_down_sync(0xffffffffu, pacc_re, off) : 0.0;
        const double pi = SP ? __shfl_down_sync(0xffffffffu, pacc_im, off) : 0.0;
        if (sub + off < L) {
            acc_re += vr; acc_im += vi;
            dacc_re += dr; dacc_im += di;
            pacc_re += pr; pacc_im += pi;
        }
#pragma unroll
        for (int r = 0; r < NRHS - 1; ++r) {
            const double xr = __shfl_down_sync(0xffffffffu, xacc_re[r], off);
            const double xi = __shfl_down_sync(0xffffffffu, xacc_im[r], off);
            if (sub + off < L) { xacc_re[r] += xr; xacc_im[r] += xi; }
        }
    }
    if (active && sub == 0) {
        auto put = [&](double *out, double *part, double re, double im) {
            double *dst = nullptr;
            if (it.part < 0) {
                if (out) dst = out + 2 * (int64_t)g.slot_tgt[it.slot_begin + j];
            } else if (part) {
                dst = part + 2 * ((int64_t)it.part + j);
            }
            if (dst) {
                dst[0] = re * kInv4Pi;
                dst[1] = im * kInv4Pi;
            }
        };
        put(ev.out_slp, ev.part_slp, acc_re, acc_im);
        if (DLP) put(ev.out_dlp, ev.part_dlp, dacc_re, dacc_im);
        if (SP) put(ev.out_sp, ev.part_sp, pacc_re, pacc_im);
#pragma unroll
        for (int r = 1; r < NRHS; ++r)
            put(ev.out_rhs[r], ev.part_slp ? ev.part_slp + r * ev.rhs_part_stride : nullptr, xacc_re[r - 1],
                xacc_im[r - 1]);
    }
}

template <bool SP, int P>
int launch_helm_p(bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    if (!tile_depth_ok(g.tile)) return (int)cudaErrorInvalidValue;
    static_assert((size_t)kWarpsPerBlock * helmholtz_tile_rows(true) * kTileMax * sizeof(double) <= kSmemNoOptIn,
                  "staging tiles fit the default shared memory");
    const size_t smem = (size_t)kWarpsPerBlock * helmholtz_tile_rows(dlp) * g.tile * sizeof(double);
    if (dlp) helmholtz_kernel<P, true, SP><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, s>>>(g, e);
    else     helmholtz_kernel<P, false, SP><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, s>>>(g, e);
    return (int)cudaGetLastError();
}

template <bool SP, int... Ps>
int dispatch_helm(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s,
                  std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_helm_p<SP, Ps>(dlp, g, e, s), 0) : 0), ...);
    return rc;
}

template <int NRHS, int P>
int launch_helm_multi_p(const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    if (!tile_depth_ok(g.tile)) return (int)cudaErrorInvalidValue;
    static_assert((size_t)kWarpsPerBlock * helmholtz_tile_rows(false, NRHS) * kTileMax * sizeof(double) <=
                      kSmemNoOptIn,
                  "staging tiles fit the default shared memory");
    const size_t smem = (size_t)kWarpsPerBlock * helmholtz_tile_rows(false, NRHS) * g.tile * sizeof(double);
    helmholtz_kernel<P, false, false, NRHS><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, s>>>(g, e);
    return (int)cudaGetLastError();
}

template <int NRHS, int... Ps>
int dispatch_helm_multi(int p, const DevGeom &g, const DevEval &e, cudaStream_t s,
                        std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_helm_multi_p<NRHS, Ps>(g, e, s), 0) : 0), ...);
    return rc;
}

}  // namespace

// Defined in helmholtz_sp.cu.
int launch_helmholtz_fp64_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s);

}  // namespace tsqbx
