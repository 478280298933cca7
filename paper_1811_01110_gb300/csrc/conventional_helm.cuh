// conventional_helm.cuh -- conventional QBX for the Helmholtz kernel (Sec.
// 2.1 eqs. local-coeffs, local-expansion with the addition theorem of
// Appendix A), FP64: the complex counterpart of conventional.cuh.
//
// P2QBXL, for a center c and the sources on its group's list, d = s - c,
// R = |d|, u = d / R:
//   M_n^m(r) = sum_s w_s mu_s h_n(kR) Re J_n^m(u),
//   M_n^m(i) = sum_s w_s mu_s h_n(kR) Im J_n^m(u),          (both complex)
// with J the angular harmonics of conventional.cuh at r = 1 (J_0^0 = 1,
// J_m^m = eta J_{m-1}^{m-1}, J_{m+1}^m = zeta J_m^m, J_n^m = zeta J_{n-1}^m
// - eps_n^m J_{n-2}^m, zeta = u_z, eta = u_x + i u_y), so that P_n^m(cos th)
// e^{im ph} = (2n-1)!!/(n-m)! J_n^m.  h_n(kR) = e^{ikR} g_n as in the
// target-specific kernel (one sincos per source).  The double layer adds the
// derivative along n_s: k h_n'(kR) (d.n_s)/R J + h_n dJ, dJ along
// (n_s - u (u.n_s))/R (forward mode).
//
// QBXL2P, for a target t, e = t - c, rho = |e|, v = e / rho:
//   u(t) = (ik/4pi) sum_n (2n+1) j_n(k rho) sum_m omega_n^m
//            ( Re J_n^m(v) M_n^m(r) + Im J_n^m(v) M_n^m(i) ),
//   omega_n^m = (2 - delta_m0) ((2n-1)!!)^2 / ((n+m)! (n-m)!),
// which is (ik/4pi) sum_n (2n+1) j_n h_n P_n(cos g) by eq.
// legendre-addition-identity.  S' differentiates j_n(k rho) J(v) along n_t:
// k j_n' (v.n_t) J + (j_n / rho) dJ, dJ along n_t - v (v.n_t); at rho = 0
// only n = 1 survives, (k/3) J_1^m(n_t).  Mapping as in conventional.cuh.
// Compiled for p <= kConvHelmMaxP.
#pragma once

#include "conventional.cuh"
#include "helmholtz_items.cuh"

namespace tsqbx {
namespace {

// omega_n^m / (4 pi kappa_n): the per-(n, m) weight against cj[n] = (2n+1)
// kappa_n j_n of helmholtz_target_factors
__host__ __device__ constexpr double conv_helm_weight(int n, int m)
{
    double df = 1.0;
    for (int q = 2 * n - 1; q > 1; q -= 2) df *= q;
    double fp = 1.0, fm = 1.0;
    for (int q = 2; q <= n + m; ++q) fp *= q;
    for (int q = 2; q <= n - m; ++q) fm *= q;
    return (m == 0 ? 1.0 : 2.0) * df * df / (fp * fm) * kInv4Pi / rec_kappa(n);
}

// The weights as a constant-bank table, filled at compile time (see
// c_conv_weight in the Laplace path).
struct ConvHelmWeightTable {
    double w[kConvHelmMaxP + 1][kConvHelmMaxP + 1];
};
constexpr ConvHelmWeightTable conv_helm_weight_table()
{
    ConvHelmWeightTable t{};
    for (int n = 0; n <= kConvHelmMaxP; ++n)
        for (int m = 0; m <= n; ++m) t.w[n][m] = conv_helm_weight(n, m);
    return t;
}
__constant__ ConvHelmWeightTable c_conv_helm_weight = conv_helm_weight_table();

// The (n, m) triangle of one source: parts per (n, m) in column order:
// single layer Re(B Jr), Im(B Jr) [, Re(B Ji), Im(B Ji) if m > 0], then the
// double layer's four (or two) in the same pattern.
template <int P, bool CS, bool CD, class Sink>
__device__ __forceinline__ void conv_helm_source(double x, double y, double z, double k, double2 wm, double nx,
                                                 double ny, double nz, Sink &sink)
{
    const double R2 = fma(x, x, fma(y, y, z * z));
    const double rinv = rsqrt(R2);
    const double ux = x * rinv, uy = y * rinv, uz = z * rinv;
    const double w = rinv / k;                          // 1/(kR)
    double sn, cs;
    sincos(k * (R2 * rinv), &sn, &cs);
    // B_n = w mu h_n(kR), h_n = e^{ikR} g_n; Bd_n = w mu k h_n'(kR) (d.n)/R
    double Br[P + 1], Bi[P + 1], Bdr[CD ? P + 1 : 1], Bdi[CD ? P + 1 : 1];
    {
        double g0r = 0.0, g0i = -w, g1r = -w, g1i = -w * w;   // g_{n-1}, g_n from n = 1
        double gr[P + 2], gi[P + 2];
        gr[0] = g0r; gi[0] = g0i;
        gr[1] = g1r; gi[1] = g1i;
#pragma unroll
        for (int n = 1; n <= P; ++n) {
            const double t = (2.0 * n + 1.0) * w;
            gr[n + 1] = fma(t, gr[n], -gr[n - 1]);
            gi[n + 1] = fma(t, gi[n], -gi[n - 1]);
        }
        // e^{iz} (w mu): combined phase and weight
        const double pr = fma(cs, wm.x, -sn * wm.y), pi = fma(cs, wm.y, sn * wm.x);
#pragma unroll
        for (int n = 0; n <= P; ++n) {
            Br[n] = fma(pr, gr[n], -pi * gi[n]);
            Bi[n] = fma(pr, gi[n], pi * gr[n]);
        }
        if (CD) {
            const double dn = fma(x, nx, fma(y, ny, z * nz)) * rinv;
            const double kd = k * dn;
#pragma unroll
            for (int n = 0; n <= P; ++n) {
                // g'_n = g_{n-1} - (n+1) w g_n, g'_0 = -g_1
                const double ddr = n == 0 ? -gr[1] : fma(-(n + 1.0) * w, gr[n], gr[n - 1]);
                const double ddi = n == 0 ? -gi[1] : fma(-(n + 1.0) * w, gi[n], gi[n - 1]);
                Bdr[CD ? n : 0] = kd * fma(pr, ddr, -pi * ddi);
                Bdi[CD ? n : 0] = kd * fma(pr, ddi, pi * ddr);
            }
        }
    }
    // angular derivative direction (n - u (u.n)) / R
    double vz = 0.0, vx = 0.0, vy = 0.0;
    if (CD) {
        const double un = fma(ux, nx, fma(uy, ny, uz * nz));
        vx = (nx - ux * un) * rinv;
        vy = (ny - uy * un) * rinv;
        vz = (nz - uz * un) * rinv;
    }
    int kk = 0;
    auto emit = [&](int n, double jr, double ji, double tr, double ti, bool cplx) {
        if (CS) {
            sink.put(kk++, Br[n] * jr);
            sink.put(kk++, Bi[n] * jr);
            if (cplx) { sink.put(kk++, Br[n] * ji); sink.put(kk++, Bi[n] * ji); }
        }
        if (CD) {
            const int c = CD ? n : 0;
            sink.put(kk++, fma(Bdr[c], jr, Br[n] * tr));
            sink.put(kk++, fma(Bdi[c], jr, Bi[n] * tr));
            if (cplx) {
                sink.put(kk++, fma(Bdr[c], ji, Br[n] * ti));
                sink.put(kk++, fma(Bdi[c], ji, Bi[n] * ti));
            }
        }
    };
    {                                                   // m = 0: real
        double Jm2 = 0.0, Jm1 = 1.0, Tm2 = 0.0, Tm1 = 0.0;
        emit(0, Jm1, 0.0, Tm1, 0.0, false);
#pragma unroll
        for (int n = 1; n <= P; ++n) {
            double Jn, Tn = 0.0;
            if (n == 1) {
                Jn = uz;
                if (CD) Tn = vz;
            } else {
                Jn = fma(uz, Jm1, -conv_eps(n, 0) * Jm2);
                if (CD) Tn = fma(vz, Jm1, fma(uz, Tm1, -conv_eps(n, 0) * Tm2));
            }
            emit(n, Jn, 0.0, Tn, 0.0, false);
            Jm2 = Jm1; Jm1 = Jn; Tm2 = Tm1; Tm1 = Tn;
        }
    }
    double Dr = 1.0, Di = 0.0, D1r = 0.0, D1i = 0.0;
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        const double nDr = fma(ux, Dr, -uy * Di), nDi = fma(ux, Di, uy * Dr);
        if (CD) {
            const double nD1r = fma(vx, Dr, -vy * Di) + fma(ux, D1r, -uy * D1i);
            const double nD1i = fma(vx, Di, vy * Dr) + fma(ux, D1i, uy * D1r);
            D1r = nD1r; D1i = nD1i;
        }
        Dr = nDr; Di = nDi;
        double Jr2 = 0.0, Ji2 = 0.0, Jr1 = Dr, Ji1 = Di;
        double Tr2 = 0.0, Ti2 = 0.0, Tr1 = D1r, Ti1 = D1i;
        emit(m, Jr1, Ji1, Tr1, Ti1, true);
#pragma unroll
        for (int n = m + 1; n <= P; ++n) {
            double Jr, Ji, Tr = 0.0, Ti = 0.0;
            if (n == m + 1) {
                Jr = uz * Jr1; Ji = uz * Ji1;
                if (CD) { Tr = fma(vz, Jr1, uz * Tr1); Ti = fma(vz, Ji1, uz * Ti1); }
            } else {
                const double ce = conv_eps(n, m);
                Jr = fma(uz, Jr1, -ce * Jr2);
                Ji = fma(uz, Ji1, -ce * Ji2);
                if (CD) {
                    Tr = fma(vz, Jr1, fma(uz, Tr1, -ce * Tr2));
                    Ti = fma(vz, Ji1, fma(uz, Ti1, -ce * Ti2));
                }
            }
            emit(n, Jr, Ji, Tr, Ti, true);
            Jr2 = Jr1; Ji2 = Ji1; Jr1 = Jr; Ji1 = Ji;
            Tr2 = Tr1; Ti2 = Ti1; Tr1 = Tr; Ti1 = Ti;
        }
    }
}

template <int P, bool CS, bool CD>
__global__ void __launch_bounds__(kConvWarps * 32)
p2qbxl_helm_kernel(const DevGeom g, const DevEval ev)
{
    constexpr int NC = 2 * (P + 1) * (P + 1) * (int(CS) + int(CD));
    __shared__ double buf_all[kConvWarps][32 * 33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kConvWarps + warp;
    if (item >= g.n_conv_items) return;
    const ConvItem it = g.conv_items[item];
    const ConvCenter cc = g.conv_centers[it.center];
    const double4_32a c = g.slot_c[cc.slot_begin];
    double *dst = ev.conv_coef + (int64_t)it.part * NC;
    for (int i = lane; i < NC; i += 32) dst[i] = 0.0;
    __syncwarp();
    ListWalk walk(g, cc.group);
    PartSink<NC> sink{buf_all[warp], dst, lane};
    for (int base = it.src_lo; base < it.src_hi; base += 32) {
        const int kq = base + lane;
        double x = 1.0, y = 0.0, z = 0.0, nx = 0.0, ny = 0.0, nz = 0.0;
        double2 wm = make_double2(0.0, 0.0);
        if (kq < it.src_hi) {
            const int s = walk.at(kq);
            if ((unsigned)s >= (unsigned)g.n_src) {
                atomicOr(ev.status, 1);
            } else {
                const double4_32a pw = g.src_pw[s];
                x = pw.x - c.x; y = pw.y - c.y; z = pw.z - c.z;
                wm = ev.wmu_c[s];
                if (CD) { const double4_32a n = g.src_n[s]; nx = n.x; ny = n.y; nz = n.z; }
            }
        }
        conv_helm_source<P, CS, CD>(x, y, z, ev.k, wm, nx, ny, nz, sink);
    }
}

constexpr int kConvHelmEvalWarps = 4;

template <int P, bool CS, bool CD, bool SP>
__global__ void __launch_bounds__(kConvHelmEvalWarps * 32)
qbxl2p_helm_kernel(const DevGeom g, const DevEval ev)
{
    constexpr int NC = 2 * (P + 1) * (P + 1) * (int(CS) + int(CD));
    __shared__ double M_all[kConvHelmEvalWarps][NC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kConvHelmEvalWarps + warp;
    if (item >= g.n_conv_eval) return;
    const ConvEvalItem it = g.conv_eval[item];
    const ConvCenter cc = g.conv_centers[it.center];
    double *M = M_all[warp];
    for (int i = lane; i < NC; i += 32) {
        double sum = 0.0;
        for (int sl = 0; sl < cc.n_slices; ++sl) sum += ev.conv_coef[(int64_t)(cc.part0 + sl) * NC + i];
        M[i] = sum;
    }
    __syncwarp();
    const bool active = lane < it.n_tgt;
    const int slot = it.slot_begin + (active ? lane : 0);
    const double4_32a e = g.slot_e[slot];
    const double k = ev.k;
    const double rho = sqrt(e.w);
    const double rhoinv = rho > 0.0 ? 1.0 / rho : 0.0;
    double vx = 0.0, vy = 0.0, vz = 1.0;                 // target direction (arbitrary at rho = 0)
    if (rho > 0.0) { vx = e.x * rhoinv; vy = e.y * rhoinv; vz = e.z * rhoinv; }
    double tx = 0.0, ty = 0.0, tz = 0.0, tdot = 0.0, wx = 0.0, wy = 0.0, wz = 0.0;
    if (SP) {
        const double4_32a tn = g.slot_n[slot];
        tx = tn.x; ty = tn.y; tz = tn.z;
        tdot = rho > 0.0 ? fma(vx, tx, fma(vy, ty, vz * tz)) : 0.0;
        wx = tx - vx * tdot; wy = ty - vy * tdot; wz = tz - vz * tdot;   // dv along n_t, times rho
    }
    double cj[P + 1];
    double caj[SP ? P + 1 : 1];
    helmholtz_target_factors<P, SP>(k, rho, tdot, cj, caj);
    const bool at_center = !(rho > 0.0);
    double usr = 0.0, usi = 0.0, udr = 0.0, udi = 0.0, upr = 0.0, upi = 0.0;
    int kk = 0;
    auto take = [&](int n, int m, double jr, double ji, double tr, double ti) {
        const double wgt = c_conv_helm_weight.w[n][m];
        const double a = wgt * cj[n];
        if (CS) {
            const double m0r = M[kk++], m0i = M[kk++];                 // M(r)
            const double m1r = m > 0 ? M[kk++] : 0.0, m1i = m > 0 ? M[kk++] : 0.0;   // M(i)
            const double dr = fma(jr, m0r, ji * m1r), di = fma(jr, m0i, ji * m1i);
            usr = fma(a, dr, usr);
            usi = fma(a, di, usi);
            if (SP) {
                // k j_n' (v.n_t) J + (j_n / rho) dJ ; at rho = 0: n = 1 only, (k/3) J_1^m(n_t)
                const double b = wgt * caj[SP ? n : 0];
                const double er = fma(tr, m0r, ti * m1r), ei = fma(tr, m0i, ti * m1i);
                upr = fma(b, dr, fma(a * rhoinv, er, upr));
                upi = fma(b, di, fma(a * rhoinv, ei, upi));
                if (at_center && n == 1) {
                    const double j1r = m == 0 ? tz : tx, j1i = m == 0 ? 0.0 : ty;
                    const double c3 = wgt * rec_kappa(1) * 3.0 * (k / 3.0);
                    upr = fma(c3, fma(j1r, m0r, j1i * m1r), upr);
                    upi = fma(c3, fma(j1r, m0i, j1i * m1i), upi);
                }
            }
        }
        if (CD) {
            const double m0r = M[kk++], m0i = M[kk++];
            const double m1r = m > 0 ? M[kk++] : 0.0, m1i = m > 0 ? M[kk++] : 0.0;
            udr = fma(a, fma(jr, m0r, ji * m1r), udr);
            udi = fma(a, fma(jr, m0i, ji * m1i), udi);
        }
    };
    {                                                   // m = 0
        double Jm2 = 0.0, Jm1 = 1.0, Tm2 = 0.0, Tm1 = 0.0;
        take(0, 0, Jm1, 0.0, Tm1, 0.0);
#pragma unroll
        for (int n = 1; n <= P; ++n) {
            double Jn, Tn = 0.0;
            if (n == 1) {
                Jn = vz;
                if (SP) Tn = wz;
            } else {
                Jn = fma(vz, Jm1, -conv_eps(n, 0) * Jm2);
                if (SP) Tn = fma(wz, Jm1, fma(vz, Tm1, -conv_eps(n, 0) * Tm2));
            }
            take(n, 0, Jn, 0.0, Tn, 0.0);
            Jm2 = Jm1; Jm1 = Jn; Tm2 = Tm1; Tm1 = Tn;
        }
    }
    double Dr = 1.0, Di = 0.0, D1r = 0.0, D1i = 0.0;
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        const double nDr = fma(vx, Dr, -vy * Di), nDi = fma(vx, Di, vy * Dr);
        if (SP) {
            const double nD1r = fma(wx, Dr, -wy * Di) + fma(vx, D1r, -vy * D1i);
            const double nD1i = fma(wx, Di, wy * Dr) + fma(vx, D1i, vy * D1r);
            D1r = nD1r; D1i = nD1i;
        }
        Dr = nDr; Di = nDi;
        double Jr2 = 0.0, Ji2 = 0.0, Jr1 = Dr, Ji1 = Di;
        double Tr2 = 0.0, Ti2 = 0.0, Tr1 = D1r, Ti1 = D1i;
        take(m, m, Jr1, Ji1, Tr1, Ti1);
#pragma unroll
        for (int n = m + 1; n <= P; ++n) {
            double Jr, Ji, Tr = 0.0, Ti = 0.0;
            if (n == m + 1) {
                Jr = vz * Jr1; Ji = vz * Ji1;
                if (SP) { Tr = fma(wz, Jr1, vz * Tr1); Ti = fma(wz, Ji1, vz * Ti1); }
            } else {
                const double ce = conv_eps(n, m);
                Jr = fma(vz, Jr1, -ce * Jr2);
                Ji = fma(vz, Ji1, -ce * Ji2);
                if (SP) {
                    Tr = fma(wz, Jr1, fma(vz, Tr1, -ce * Tr2));
                    Ti = fma(wz, Ji1, fma(vz, Ti1, -ce * Ti2));
                }
            }
            take(n, m, Jr, Ji, Tr, Ti);
            Jr2 = Jr1; Ji2 = Ji1; Jr1 = Jr; Ji1 = Ji;
            Tr2 = Tr1; Ti2 = Ti1; Tr1 = Tr; Ti1 = Ti;
        }
    }
    if (active) {
        // times ik: (x + iy) ik = (-k y, k x)
        const int64_t t = g.slot_tgt[slot];
        if (CS && ev.out_slp) { ev.out_slp[2 * t] = -k * usi; ev.out_slp[2 * t + 1] = k * usr; }
        if (CD && ev.out_dlp) { ev.out_dlp[2 * t] = -k * udi; ev.out_dlp[2 * t + 1] = k * udr; }
        if (SP && ev.out_sp) { ev.out_sp[2 * t] = -k * upi; ev.out_sp[2 * t + 1] = k * upr; }
    }
}

template <int P, bool CS, bool CD, bool SP>
int launch_conv_helm_p(const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (g.n_conv_items > 0) {
        const int64_t blocks = (g.n_conv_items + kConvWarps - 1) / kConvWarps;
        p2qbxl_helm_kernel<P, CS, CD><<<(unsigned)blocks, kConvWarps * 32, 0, s>>>(g, e);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return (int)err;
    }
    if (g.n_conv_eval > 0) {
        const int64_t blocks = (g.n_conv_eval + kConvHelmEvalWarps - 1) / kConvHelmEvalWarps;
        qbxl2p_helm_kernel<P, CS, CD, SP><<<(unsigned)blocks, kConvHelmEvalWarps * 32, 0, s>>>(g, e);
    }
    return (int)cudaGetLastError();
}

template <int P>
int launch_conv_helm_layers(unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const bool cs = (layers & 5u) != 0, cd = (layers & 2u) != 0, sp = (layers & 4u) != 0;
    if (cs && cd) return sp ? launch_conv_helm_p<P, true, true, true>(g, e, s) : launch_conv_helm_p<P, true, true, false>(g, e, s);
    if (cs) return sp ? launch_conv_helm_p<P, true, false, true>(g, e, s) : launch_conv_helm_p<P, true, false, false>(g, e, s);
    if (cd) return launch_conv_helm_p<P, false, true, false>(g, e, s);
    return (int)cudaErrorInvalidValue;
}

template <int... Ps>
int dispatch_conv_helm(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s,
                       std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_conv_helm_layers<Ps>(layers, g, e, s), 0) : 0), ...);
    return rc;
}

template <int LO, int HI>
int launch_conv_helm_range(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return dispatch_conv_helm(p, layers, g, e, s, offset_seq<LO>(std::make_integer_sequence<int, HI - LO + 1>{}));
}

}  // namespace

// Order ranges, one per translation unit (conventional_helm_pLO_HI.cu).
int launch_conv_helm_p0_8(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conv_helm_p9_10(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conv_helm_p11_12(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);

}  // namespace tsqbx
