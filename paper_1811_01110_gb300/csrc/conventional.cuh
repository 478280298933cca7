// conventional.cuh -- conventional QBX for centers with many targets (Sec. 2.1
// eqs. local-coeffs, local-expansion, laplace-identity; which centers take
// this path is decided by the cost model of Table 2, in plan.cu).  Laplace,
// FP64.
//
// P2QBXL (coefficient formation), for a center c and the sources s on its
// group's list, d = s - c:
//   M_n^m = sum_s w_s mu_s J_n^m(d),  0 <= m <= n <= p,  complex,
// with J the irregular solid harmonics I_n^m(d) = (n-m)! P_n^m(cos th) e^{im ph}
// / |d|^{n+1} scaled by (2n-1)!!  (P_n^m without the Condon-Shortley phase,
// which cancels below).  From (n-m) P_n^m = (2n-1) x P_{n-1}^m - (n+m-1)
// P_{n-2}^m and P_m^m = (2m-1)!! sin^m (DLMF 14.10.3, 14.7.15):
//   J_0^0 = 1/r, J_m^m = eta J_{m-1}^{m-1}, J_{m+1}^m = zeta J_m^m,
//   J_n^m = zeta J_{n-1}^m - eps_n^m a J_{n-2}^m,
//   a = 1/r^2, zeta = z a, eta = (x + i y) a, eps_n^m = (n+m-1)(n-m-1)/((2n-1)(2n-3)).
// The double layer forms the derivative of M along n_s (forward mode).
//
// QBXL2P (evaluation), for a target t of c, e = t - c:
//   u(t) = (1/4pi) sum_{n<=p} sum_{m=0}^n (2 - delta_m0) (2n-1)!! tau_n^m
//            Re( K_n^m(e) conj(M_n^m) )
// with the regular solid harmonics r^n P_n^m e^{im ph} / (n+m)! = tau_n^m K_n^m:
//   K_0^0 = 1, K_m^m = xi K_{m-1}^{m-1}, K_{m+1}^m = z K_m^m,
//   K_n^m = z K_{n-1}^m - eps_n^m r^2 K_{n-2}^m,  xi = x + i y,
//   tau_m^m = 1/(2^m m!), tau_n^m = tau_{n-1}^m (2n-1)/((n-m)(n+m)).
// By the addition theorem (eq. legendre-addition-identity) the inner sum over
// m is |e|^n / |d|^{n+1} P_n(cos g): u is the truncated expansion the
// target-specific kernels evaluate (eq. tsqbx).  S' differentiates K along n_t.
//
// Mapping.  P2QBXL: one warp per (center, source slice); lane l takes every
// 32nd source and walks its whole (n, m) triangle in registers, storing each
// coefficient part to its row of a padded shared buffer; every 32 parts, lane
// l adds up column l (the 32 sources' contributions to one part) into the
// slice's partial block.  QBXL2P: one warp per (center, up to 32
// targets); the center's partial blocks are summed in slice order into shared
// memory, one lane per target.  Every sum runs in a fixed order, so results
// are deterministic.
#pragma once

#include <utility>

#include "internal.cuh"

namespace tsqbx {
namespace {

constexpr int kConvWarps = 4;

template <int LO, int... Is>
constexpr std::integer_sequence<int, (LO + Is)...> offset_seq(std::integer_sequence<int, Is...>)
{
    return {};
}

__host__ __device__ constexpr double conv_eps(int n, int m)
{
    return (1.0 * (n + m - 1) * (n - m - 1)) / ((2.0 * n - 1.0) * (2.0 * n - 3.0));
}

// (2 - delta_m0) (2n-1)!! tau_n^m / (4 pi)
__host__ __device__ constexpr double conv_weight(int n, int m)
{
    double t = 1.0;
    for (int j = 1; j <= m; ++j) t /= 2.0 * j;
    for (int j = m + 1; j <= n; ++j) t *= (2.0 * j - 1.0) / ((double)(j - m) * (double)(j + m));
    double df = 1.0;
    for (int q = 2 * n - 1; q > 1; q -= 2) df *= q;
    return (m == 0 ? 1.0 : 2.0) * df * t * kInv4Pi;
}

// The weights as a constant-bank table, filled at compile time: indexed by the
// (n, m) of the unrolled triangles, each is an immediate constant-bank operand.
struct ConvWeightTable {
    double w[21][21];
};
constexpr ConvWeightTable conv_weight_table()
{
    ConvWeightTable t{};
    for (int n = 0; n <= 20; ++n)
        for (int m = 0; m <= n; ++m) t.w[n][m] = conv_weight(n, m);
    return t;
}
__constant__ ConvWeightTable c_conv_weight = conv_weight_table();

// Receives the coefficient parts of one source per lane, in order: part k of
// lane l goes to row l, column k mod 32 of the warp's padded 32 x 33 buffer;
// after every 32 parts (and at the end) lane l adds up column l over the 32
// rows (a fixed order) into the item's partial block, dst[32 (k / 32) + l].
// One shared store per part keeps the unrolled (n, m) triangles short.
template <int NC>
struct PartSink {
    double *buf;     // the warp's 32 x 33 doubles
    double *dst;     // the item's NC partial coefficients (zeroed)
    int lane;
    __device__ __forceinline__ void put(int k, double x)
    {
        buf[33 * lane + (k & 31)] = x;
        if ((k & 31) == 31 || k == NC - 1) {
            if (k == NC - 1) {
#pragma unroll
                for (int i = (k & 31) + 1; i < 32; ++i) buf[33 * lane + i] = 0.0;
            }
            __syncwarp();
            double sum = 0.0;
#pragma unroll 1
            for (int r = 0; r < 32; ++r) sum += buf[33 * r + lane];
            const int at = (k & ~31) + lane;
            if (at < NC) dst[at] += sum;
            __syncwarp();
        }
    }
};

// The (n, m) triangle of one source, w mu folded into the seed; parts go to
// the sink as, per (n, m) in column order (m = 0, n = 0..p; m = 1, n = 1..p;
// ...): single layer re [, im if m > 0], then double layer re [, im].
template <int P, bool CS, bool CD, class Sink>
__device__ __forceinline__ void conv_source(double x, double y, double z, double wm, double nx, double ny,
                                            double nz, Sink &sink)
{
    const double r2 = fma(x, x, fma(y, y, z * z));
    const double rinv = rsqrt(r2);
    const double a = rinv * rinv;
    const double zeta = z * a, er = x * a, ei = y * a;
    double a1 = 0.0, zeta1 = 0.0, er1 = 0.0, ei1 = 0.0, seed1 = 0.0;
    if (CD) {                                   // derivatives along n_s
        const double dn = fma(x, nx, fma(y, ny, z * nz));
        a1 = -2.0 * dn * a * a;
        zeta1 = fma(nz, a, z * a1);
        er1 = fma(nx, a, x * a1);
        ei1 = fma(ny, a, y * a1);
        seed1 = -wm * dn * a * rinv;
    }
    const double seed = wm * rinv;
    int k = 0;
    auto emit = [&](double jr, double ji, double tr, double ti, bool cplx) {
        if (CS) { sink.put(k++, jr); if (cplx) sink.put(k++, ji); }
        if (CD) { sink.put(k++, tr); if (cplx) sink.put(k++, ti); }
    };
    // m = 0 column: real
    {
        double Jm2 = 0.0, Jm1 = seed, Tm2 = 0.0, Tm1 = seed1;
        emit(Jm1, 0.0, Tm1, 0.0, false);
#pragma unroll
        for (int n = 1; n <= P; ++n) {
            double Jn, Tn = 0.0;
            if (n == 1) {
                Jn = zeta * Jm1;
                if (CD) Tn = fma(zeta1, Jm1, zeta * Tm1);
            } else {
                const double ea = conv_eps(n, 0) * a;
                Jn = fma(zeta, Jm1, -ea * Jm2);
                if (CD) Tn = fma(zeta1, Jm1, zeta * Tm1) - conv_eps(n, 0) * fma(a1, Jm2, a * Tm2);
            }
            emit(Jn, 0.0, Tn, 0.0, false);
            Jm2 = Jm1; Jm1 = Jn; Tm2 = Tm1; Tm1 = Tn;
        }
    }
    // columns m >= 1 from the diagonal J_m^m = eta J_{m-1}^{m-1}
    double Dr = seed, Di = 0.0, D1r = seed1, D1i = 0.0;
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        const double nDr = fma(er, Dr, -ei * Di), nDi = fma(er, Di, ei * Dr);
        if (CD) {
            const double nD1r = fma(er1, Dr, -ei1 * Di) + fma(er, D1r, -ei * D1i);
            const double nD1i = fma(er1, Di, ei1 * Dr) + fma(er, D1i, ei * D1r);
            D1r = nD1r; D1i = nD1i;
        }
        Dr = nDr; Di = nDi;
        double Jr2 = 0.0, Ji2 = 0.0, Jr1 = Dr, Ji1 = Di;
        double Tr2 = 0.0, Ti2 = 0.0, Tr1 = D1r, Ti1 = D1i;
        emit(Jr1, Ji1, Tr1, Ti1, true);
#pragma unroll
        for (int n = m + 1; n <= P; ++n) {
            double Jr, Ji, Tr = 0.0, Ti = 0.0;
            if (n == m + 1) {
                Jr = zeta * Jr1; Ji = zeta * Ji1;
                if (CD) { Tr = fma(zeta1, Jr1, zeta * Tr1); Ti = fma(zeta1, Ji1, zeta * Ti1); }
            } else {
                const double ea = conv_eps(n, m) * a;
                Jr = fma(zeta, Jr1, -ea * Jr2);
                Ji = fma(zeta, Ji1, -ea * Ji2);
                if (CD) {
                    Tr = fma(zeta1, Jr1, zeta * Tr1) - conv_eps(n, m) * fma(a1, Jr2, a * Tr2);
                    Ti = fma(zeta1, Ji1, zeta * Ti1) - conv_eps(n, m) * fma(a1, Ji2, a * Ti2);
                }
            }
            emit(Jr, Ji, Tr, Ti, true);
            Jr2 = Jr1; Ji2 = Ji1; Jr1 = Jr; Ji1 = Ji;
            Tr2 = Tr1; Ti2 = Ti1; Tr1 = Tr; Ti1 = Ti;
        }
    }
}

template <int P, bool CS, bool CD>
__global__ void __launch_bounds__(kConvWarps * 32)
p2qbxl_kernel(const DevGeom g, const DevEval ev)
{
    constexpr int NC = (P + 1) * (P + 1) * (int(CS) + int(CD));
    __shared__ double buf_all[kConvWarps][32 * 33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kConvWarps + warp;
    if (item >= g.n_conv_items) return;                  // whole warp leaves together
    const ConvItem it = g.conv_items[item];
    const ConvCenter cc = g.conv_centers[it.center];
    const double4_32a c = g.slot_c[cc.slot_begin];
    double *dst = ev.conv_coef + (int64_t)it.part * NC;
    for (int i = lane; i < NC; i += 32) dst[i] = 0.0;
    __syncwarp();
    ListWalk walk(g, cc.group);
    PartSink<NC> sink{buf_all[warp], dst, lane};
    for (int base = it.src_lo; base < it.src_hi; base += 32) {
        const int k = base + lane;
        double x = 1.0, y = 0.0, z = 0.0, wm = 0.0, nx = 0.0, ny = 0.0, nz = 0.0;
        if (k < it.src_hi) {
            const int s = walk.at(k);
            if ((unsigned)s >= (unsigned)g.n_src) {
                atomicOr(ev.status, 1);
            } else {
                const double4_32a pw = g.src_pw[s];
                x = pw.x - c.x; y = pw.y - c.y; z = pw.z - c.z;
                wm = ev.wmu[s];
                if (CD) { const double4_32a n = g.src_n[s]; nx = n.x; ny = n.y; nz = n.z; }
            }
        }
        conv_source<P, CS, CD>(x, y, z, wm, nx, ny, nz, sink);
    }
}

template <int P, bool CS, bool CD, bool SP>
__global__ void __launch_bounds__(kConvWarps * 32)
qbxl2p_kernel(const DevGeom g, const DevEval ev)
{
    constexpr int NC = (P + 1) * (P + 1) * (int(CS) + int(CD));
    __shared__ double M_all[kConvWarps][NC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kConvWarps + warp;
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
    const double x = e.x, y = e.y, z = e.z, r2 = e.w;
    double zx = 0.0, zy = 0.0, zz = 0.0, q1 = 0.0;       // n_t and d(r^2) along n_t
    if (SP) {
        const double4_32a tn = g.slot_n[slot];
        zx = tn.x; zy = tn.y; zz = tn.z;
        q1 = 2.0 * fma(x, zx, fma(y, zy, z * zz));
    }
    double us = 0.0, ud = 0.0, up = 0.0;
    int k = 0;
    auto take = [&](int n, int m, double kr, double ki, double k1r, double k1i) {
        const double w = c_conv_weight.w[n][m];
        if (CS) {
            const double mr = M[k++], mi = m > 0 ? M[k++] : 0.0;
            us = fma(w, fma(kr, mr, ki * mi), us);
            if (SP) up = fma(w, fma(k1r, mr, k1i * mi), up);
        }
        if (CD) {
            const double mr = M[k++], mi = m > 0 ? M[k++] : 0.0;
            ud = fma(w, fma(kr, mr, ki * mi), ud);
        }
    };
    // m = 0 column: real
    {
        double Km2 = 0.0, Km1 = 1.0, Tm2 = 0.0, Tm1 = 0.0;
        take(0, 0, Km1, 0.0, Tm1, 0.0);
#pragma unroll
        for (int n = 1; n <= P; ++n) {
            double Kn, Tn = 0.0;
            if (n == 1) {
                Kn = z * Km1;
                if (SP) Tn = fma(zz, Km1, z * Tm1);
            } else {
                const double er2 = conv_eps(n, 0) * r2;
                Kn = fma(z, Km1, -er2 * Km2);
                if (SP) Tn = fma(zz, Km1, z * Tm1) - conv_eps(n, 0) * fma(q1, Km2, r2 * Tm2);
            }
            take(n, 0, Kn, 0.0, Tn, 0.0);
            Km2 = Km1; Km1 = Kn; Tm2 = Tm1; Tm1 = Tn;
        }
    }
    double Dr = 1.0, Di = 0.0, D1r = 0.0, D1i = 0.0;
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        const double nDr = fma(x, Dr, -y * Di), nDi = fma(x, Di, y * Dr);
        if (SP) {
            const double nD1r = fma(zx, Dr, -zy * Di) + fma(x, D1r, -y * D1i);
            const double nD1i = fma(zx, Di, zy * Dr) + fma(x, D1i, y * D1r);
            D1r = nD1r; D1i = nD1i;
        }
        Dr = nDr; Di = nDi;
        double Kr2 = 0.0, Ki2 = 0.0, Kr1 = Dr, Ki1 = Di;
        double Tr2 = 0.0, Ti2 = 0.0, Tr1 = D1r, Ti1 = D1i;
        take(m, m, Kr1, Ki1, Tr1, Ti1);
#pragma unroll
        for (int n = m + 1; n <= P; ++n) {
            double Kr, Ki, Tr = 0.0, Ti = 0.0;
            if (n == m + 1) {
                Kr = z * Kr1; Ki = z * Ki1;
                if (SP) { Tr = fma(zz, Kr1, z * Tr1); Ti = fma(zz, Ki1, z * Ti1); }
            } else {
                const double er2 = conv_eps(n, m) * r2;
                Kr = fma(z, Kr1, -er2 * Kr2);
                Ki = fma(z, Ki1, -er2 * Ki2);
                if (SP) {
                    Tr = fma(zz, Kr1, z * Tr1) - conv_eps(n, m) * fma(q1, Kr2, r2 * Tr2);
                    Ti = fma(zz, Ki1, z * Ti1) - conv_eps(n, m) * fma(q1, Ki2, r2 * Ti2);
                }
            }
            take(n, m, Kr, Ki, Tr, Ti);
            Kr2 = Kr1; Ki2 = Ki1; Kr1 = Kr; Ki1 = Ki;
            Tr2 = Tr1; Ti2 = Ti1; Tr1 = Tr; Ti1 = Ti;
        }
    }
    if (active) {
        const int t = g.slot_tgt[slot];
        if (CS && ev.out_slp) ev.out_slp[t] = us;
        if (CD && ev.out_dlp) ev.out_dlp[t] = ud;
        if (SP && ev.out_sp) ev.out_sp[t] = up;
    }
}

template <int P, bool CS, bool CD, bool SP>
int launch_conv_p(const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (g.n_conv_items > 0) {
        const int64_t blocks = (g.n_conv_items + kConvWarps - 1) / kConvWarps;
        p2qbxl_kernel<P, CS, CD><<<(unsigned)blocks, kConvWarps * 32, 0, s>>>(g, e);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return (int)err;
    }
    if (g.n_conv_eval > 0) {
        const int64_t blocks = (g.n_conv_eval + kConvWarps - 1) / kConvWarps;
        qbxl2p_kernel<P, CS, CD, SP><<<(unsigned)blocks, kConvWarps * 32, 0, s>>>(g, e);
    }
    return (int)cudaGetLastError();
}

template <int P>
int launch_conv_layers(unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const bool cs = (layers & 5u) != 0, cd = (layers & 2u) != 0, sp = (layers & 4u) != 0;
    if (cs && cd) return sp ? launch_conv_p<P, true, true, true>(g, e, s) : launch_conv_p<P, true, true, false>(g, e, s);
    if (cs) return sp ? launch_conv_p<P, true, false, true>(g, e, s) : launch_conv_p<P, true, false, false>(g, e, s);
    if (cd) return launch_conv_p<P, false, true, false>(g, e, s);
    return (int)cudaErrorInvalidValue;
}

template <int... Ps>
int dispatch_conv(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s,
                  std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_conv_layers<Ps>(layers, g, e, s), 0) : 0), ...);
    return rc;
}

// Instantiates orders LO..HI (one translation unit per range, compiled in
// parallel: the unrolled (n, m) triangles make high orders slow to compile).
template <int LO, int HI>
int launch_conv_range(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return dispatch_conv(p, layers, g, e, s, offset_seq<LO>(std::make_integer_sequence<int, HI - LO + 1>{}));
}

}  // namespace

// Order ranges, one per translation unit (conventional_pLO_HI.cu).
int launch_conv_p0_10(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conv_p11_13(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conv_p14_15(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conv_p16_17(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conv_p18_19(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conv_p20(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);

}  // namespace tsqbx
