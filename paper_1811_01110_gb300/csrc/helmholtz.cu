// helmholtz.cu -- Helmholtz TSQBX single-layer kernel, FP64 throughout.
//
// Appendix A:  G_k^(p)(t,s) = ik/(4pi) sum_{n<=p} (2n+1) j_n(k rho) h_n(kR) P_n(cos g)
// with rho = |t-c|, R = |s-c|, h_n = h_n^(1).
//  * per target (once per work item): j_n(k rho), n <= p, by Miller's downward
//    recurrence f_{n-1} = (2n+1)/z f_n - f_{n+1} (DLMF 10.51.1), started
//    p + 20 + ceil(z) terms up and normalised against j_0 = sin z/z or
//    j_1 = sin z/z^2 - cos z/z, whichever is larger;
//  * per pair: h_n(z) = e^{iz} g_n(z), z = kR, where g_n obeys the same
//    recurrence upwards (DLMF 10.51.1) from g_0 = -i/z, g_1 = -(1/z + i/z^2)
//    (DLMF 10.49.6 with 10.47.5), so one sincos per pair gives every order;
//  * P_n(cos g) by the scaled Bonnet recurrence with q = 1 (P_n = kappa_n T_n).
// All of it -- Bessel and Hankel recurrences and the sums -- in FP64.
#include <utility>

#include "internal.cuh"

namespace tsqbx {
namespace {

template <int P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
helmholtz_slp_kernel(const DevGeom g, const DevEval ev)
{
    __shared__ double tile[kWarpsPerBlock][5][kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    const Item it = g.items[item];
    const int L = it.L;
    const int j = lane / L, sub = lane - j * L;
    const bool active = j < it.n_tgt;
    const double k = ev.k, kinv = 1.0 / ev.k;
    double cx = 0, cy = 0, cz = 0, ex = 0, ey = 0, ez = 0, rhoinv = 0;
    double cj[P + 1];                  // (2n+1) kappa_n j_n(k rho)
#pragma unroll
    for (int n = 0; n <= P; ++n) cj[n] = 0.0;
    if (active) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double4_32a e = g.slot_e[it.slot_begin + j];
        cx = c.x; cy = c.y; cz = c.z;
        ex = e.x; ey = e.y; ez = e.z;
        const double rho = sqrt(e.w);
        rhoinv = rho > 0.0 ? 1.0 / rho : 0.0;
        const double z = k * rho;
        double jn[P + 1];
        if (z == 0.0) {
            jn[0] = 1.0;
#pragma unroll
            for (int n = 1; n <= P; ++n) jn[n] = 0.0;
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
            jn[P] = fb;
            if (P >= 1) jn[P >= 1 ? P - 1 : 0] = (2.0 * P + 1.0) * zinv * fb - fa;
#pragma unroll
            for (int n = P - 1; n >= 1; --n) {
                jn[n - 1] = (2.0 * n + 1.0) * zinv * jn[n] - jn[n + 1];
                if (fabs(jn[n - 1]) > 1e200) {
#pragma unroll
                    for (int m = 0; m <= P; ++m)
                        if (m >= n - 1) jn[m] *= 1e-200;
                }
            }
            double sn, cs;
            sincos(z, &sn, &cs);
            const double j0 = sn * zinv;
            const double j1 = (sn * zinv - cs) * zinv;
            const double scale = (P >= 1 && fabs(j1) > fabs(j0)) ? j1 / jn[P >= 1 ? 1 : 0]
                                                                 : j0 / jn[0];
#pragma unroll
            for (int n = 0; n <= P; ++n) jn[n] *= scale;
        }
#pragma unroll
        for (int n = 0; n <= P; ++n) cj[n] = (2.0 * n + 1.0) * rec_kappa(n) * jn[n];
    }
    const int64_t s0 = g.grp_off[it.group];
    const int src_hi = it.src_hi;
    double (*T)[kTile] = tile[warp];
    double acc_re = 0.0, acc_im = 0.0;

    for (int base = it.src_lo; base < src_hi; base += kTile) {
        const int cnt = min(kTile, src_hi - base);
        for (int kk = lane; kk < cnt; kk += 32) {
            int s = g.grp_src[s0 + base + kk];
            double2 wm = make_double2(0.0, 0.0);
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu_c[s];
            const double4_32a pw = g.src_pw[s];
            T[0][kk] = pw.x; T[1][kk] = pw.y; T[2][kk] = pw.z;
            T[3][kk] = wm.x; T[4][kk] = wm.y;
        }
        __syncwarp();
        if (active) {
            for (int kk = sub; kk < cnt; kk += L) {
                const double dx = T[0][kk] - cx, dy = T[1][kk] - cy, dz = T[2][kk] - cz;
                const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const double rinv = rsqrt(R2);
                const double x = fma(dx, ex, fma(dy, ey, dz * ez)) * rinv * rhoinv;
                const double w = rinv * kinv;               // 1/z
                const double z = k * (R2 * rinv);
                // n = 0: g_0 = (0, -w)
                double A = 0.0, B = -cj[0] * w;
                double gmr = 0.0, gmi = -w;                 // g_{n-1}
                double gr = -w, gi = -w * w;                // g_n (n = 1)
                double Tm = 1.0, Tc = x;                    // T_{n-1}, T_n
                if (P >= 1) {
                    const double c1 = cj[1] * x;
                    A = fma(c1, gr, A);
                    B = fma(c1, gi, B);
                }
#pragma unroll
                for (int n = 1; n < P; ++n) {
                    const double t = (2.0 * n + 1.0) * w;
                    const double nr = fma(t, gr, -gmr), ni = fma(t, gi, -gmi);
                    gmr = gr; gmi = gi; gr = nr; gi = ni;
                    const double Tn = fma(x, Tc, -rec_beta(n) * Tm);
                    Tm = Tc; Tc = Tn;
                    const double c = cj[n + 1] * Tn;
                    A = fma(c, gr, A);
                    B = fma(c, gi, B);
                }
                double sn, cs;
                sincos(z, &sn, &cs);
                // v = e^{iz} (A + iB);  u = ik v;  acc += u * (w mu)
                const double vr = fma(cs, A, -sn * B), vi = fma(sn, A, cs * B);
                const double ur = -k * vi, ui = k * vr;
                const double wr = T[3][kk], wi = T[4][kk];
                acc_re = fma(ur, wr, fma(-ui, wi, acc_re));
                acc_im = fma(ur, wi, fma(ui, wr, acc_im));
            }
        }
        __syncwarp();
    }
    for (int off = 1; off < L; off <<= 1) {
        const double vr = __shfl_down_sync(0xffffffffu, acc_re, off);
        const double vi = __shfl_down_sync(0xffffffffu, acc_im, off);
        if (sub + off < L) { acc_re += vr; acc_im += vi; }
    }
    if (active && sub == 0) {
        double *dst = nullptr;
        if (it.part < 0) {
            if (ev.out_slp) dst = ev.out_slp + 2 * (int64_t)g.slot_tgt[it.slot_begin + j];
        } else {
            dst = ev.part_slp + 2 * ((int64_t)it.part + j);
        }
        if (dst) {
            dst[0] = acc_re * kInv4Pi;
            dst[1] = acc_im * kInv4Pi;
        }
    }
}

template <int P>
int launch_p(const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    helmholtz_slp_kernel<P><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(g, e);
    return (int)cudaGetLastError();
}

template <int... Ps>
int dispatch(int p, const DevGeom &g, const DevEval &e, cudaStream_t s,
             std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_p<Ps>(g, e, s), 0) : 0), ...);
    return rc;
}

}  // namespace

int launch_helmholtz_fp64(int p, bool slp, bool dlp, const DevGeom &g, const DevEval &e,
                          cudaStream_t s)
{
    if (!slp || dlp) return (int)cudaErrorNotSupported;
    return dispatch(p, g, e, s, std::make_integer_sequence<int, 21>{});
}

}  // namespace tsqbx
