// laplace_items.cuh -- the per-work-item bodies of the Laplace TSQBX kernels
// (FP64 and mixed precision), shared by the one-plan kernels
// (laplace_fp64.cu, laplace_mixed.cu) and the persistent batched kernel
// (batch.cu).  The arithmetic is documented at the top of laplace_fp64.cu and
// laplace_mixed.cu.  One call processes one Item with the calling warp.
//
// Two data paths:
//  * items with several targets stage the group's sources through the warp's
//    shared-memory tile T (each staged source serves every target of the item);
//  * items with one target (a group of one center, e.g. per-center radius
//    lists) gain nothing from staging: all 32 lanes read their sources straight
//    from global memory (coalesced along the list) and combine with a full-warp
//    butterfly reduction.
#pragma once

#include "dfloat.cuh"
#include "f32x2.cuh"
#include "internal.cuh"

namespace tsqbx {

// Order forms.  A template order P >= 0 compiles one kernel per order with
// the recurrences fully unrolled and their coefficients as immediates.  P < 0
// compiles one kernel for every order: the order is the runtime value the
// pair functions receive (prt), the loops over n are unrolled by -P, and the
// coefficients are read from the constant-memory table kRec (the same values,
// so both forms compute the same quantities in the same order).
struct RecTable {
    double kappa[kPMax + 2], beta[kPMax + 2], lambda[kPMax + 2], gamma[kPMax + 2];
    float kappa_f[kPMax + 2], beta_f[kPMax + 2], lambda_f[kPMax + 2],
        gamma_f[kPMax + 2];
};
constexpr RecTable make_rec_table()
{
    RecTable t{};
    for (int n = 0; n < kPMax + 2; ++n) {
        t.kappa[n] = rec_kappa(n);
        t.beta[n] = n > 0 ? rec_beta(n) : 0.0;
        t.lambda[n] = rec_lambda(n);
        t.gamma[n] = n > 0 ? rec_gamma(n) : 0.0;
        t.kappa_f[n] = (float)t.kappa[n];
        t.beta_f[n] = (float)t.beta[n];
        t.lambda_f[n] = (float)t.lambda[n];
        t.gamma_f[n] = (float)t.gamma[n];
    }
    return t;
}
static __constant__ RecTable kRec = make_rec_table();

// for (n = lo; n < hi; ++n) step(n) and for (n = hi - 1; n >= lo; --n)
// step(n), unrolled completely for a fixed order and by -P for the
// runtime-order form.
template <int P, class F>
__device__ __forceinline__ void order_loop_up(int lo, int hi, F &&step)
{
    if constexpr (P >= 0) {
#pragma unroll
        for (int n = lo; n < hi; ++n) step(n);
    } else {
#pragma unroll (-P)
        for (int n = lo; n < hi; ++n) step(n);
    }
}
template <int P, class F>
__device__ __forceinline__ void order_loop_down(int lo, int hi, F &&step)
{
    if constexpr (P >= 0) {
#pragma unroll
        for (int n = hi - 1; n >= lo; --n) step(n);
    } else {
#pragma unroll (-P)
        for (int n = hi - 1; n >= lo; --n) step(n);
    }
}
template <int P> __device__ __forceinline__ int order_of(int prt) { return P < 0 ? prt : P; }
template <int P> __device__ __forceinline__ double c_kappa(int n) { if constexpr (P < 0) return kRec.kappa[n]; else return rec_kappa(n); }
template <int P> __device__ __forceinline__ double c_beta(int n) { if constexpr (P < 0) return kRec.beta[n]; else return rec_beta(n); }
template <int P> __device__ __forceinline__ double c_lambda(int n) { if constexpr (P < 0) return kRec.lambda[n]; else return rec_lambda(n); }
template <int P> __device__ __forceinline__ double c_gamma(int n) { if constexpr (P < 0) return kRec.gamma[n]; else return rec_gamma(n); }
template <int P> __device__ __forceinline__ float c_kappa_f(int n) { if constexpr (P < 0) return kRec.kappa_f[n]; else return (float)rec_kappa(n); }
template <int P> __device__ __forceinline__ float c_beta_f(int n) { if constexpr (P < 0) return kRec.beta_f[n]; else return (float)rec_beta(n); }
template <int P> __device__ __forceinline__ float c_lambda_f(int n) { if constexpr (P < 0) return kRec.lambda_f[n]; else return (float)rec_lambda(n); }
template <int P> __device__ __forceinline__ float c_gamma_f(int n) { if constexpr (P < 0) return kRec.gamma_f[n]; else return (float)rec_gamma(n); }

// One (target, source) pair in FP64: d = s - c, e = t - c, wm = w mu, n = n_s,
// t = n_t and ent = e.n_t (S').
//
// Single layer alone: S = sum kappa_n T_n with T_{n+1} = qx T_n - beta_n q2
// T_{n-1}, summed by Clenshaw's backward recurrence b_k = kappa_k + qx b_{k+1}
// - beta_{k+1} q2 b_{k+2}, S = b_0 (T_1 = qx T_0): three operations per order
// with the sum folded in.
//
// With the double layer or S': everything follows from the derivatives
// Q'_n = (rho/R)^{n-1} P_n'(x) alone (rec_lambda / rec_gamma recurrence, three
// operations per order plus one sum).  With S2 = sum_{n<=p} Q'_n and
// S2m = sum_{n<p} Q'_n, summing P'_{n+1} - x P'_n = (n+1) P_n and
// P'_{n+1} - P'_{n-1} = (2n+1) P_n over n <= p gives
//   S  = sum Q_n       = (1 - 2 qx + q2) S2 + Q'_{p+1} - q2 Q'_p,
//   S1 = sum (n+1) Q_n = (1 - qx) S2 + Q'_{p+1},
// and since dQ_n/dqx = Q'_n and 2 dQ_n/dq2 = -Q'_{n-1} (the identity
// x P'_n - P'_{n-1} = n P_n), with grad_s qx = (e - 2 qx d)/R^2,
// grad_s q2 = -2 q2 d/R^2, grad_t qx = d/R^2 and grad_t q2 = 2 e/R^2:
//   double layer  n_s.grad_s (S/R) = (1/R^3) [ -a S1 + (b - a qx) S2 ]
//                                  = (1/R^3) [ (b - a) S2 - a Q'_{p+1} ],
//   S'            n_t.grad_t (S/R) = (1/R^3) [ (d.n_t) S2 - (e.n_t) S2m ],
// a = d.n_s, b = e.n_s.  The closing sums cancel at most by a factor of a few
// hundred over rho/R <= 0.9, orders 0..20, a cost of ~2e-14 in FP64.
// The pair's geometry: 1/R, 1/R^2, qx = (d.e)/R^2 and q2 = rho^2/R^2.
__device__ __forceinline__ void pair_geom_fp64(double dx, double dy, double dz, double ex, double ey, double ez,
                                               double rho2, double &rinv, double &r2inv, double &qx, double &q2)
{
    const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
    rinv = rsqrt(R2);
    r2inv = rinv * rinv;
    qx = fma(dx, ex, fma(dy, ey, dz * ez)) * r2inv;
    q2 = rho2 * r2inv;
}

// The single layer's sum S = b_0 by Clenshaw's backward recurrence (order p).
template <int P>
__device__ __forceinline__ double slp_clenshaw_fp64(double qx, double q2, int p)
{
    // b_{k+1}, b_{k+2} at k = p - 2 (b_{p+1} = 0 drops out of b_{p-1})
    double b1 = p >= 1 ? fma(qx, c_kappa<P>(p), c_kappa<P>(max(p - 1, 0))) : 1.0, b2 = c_kappa<P>(p);
    order_loop_down<P>(0, p - 1, [&](int k) {
        const double bk = fma(-(c_beta<P>(k + 1) * q2), b2, fma(qx, b1, c_kappa<P>(k)));
        b2 = b1; b1 = bk;
    });
    return b1;
}

// The Q'-recurrence sums of the double layer and S' (order p): S2m = sum_{n<p}
// Q'_n, Q'_p, Q'_{p+1}, S2 = S2m + Q'_p and the single layer's S.
template <int P>
__device__ __forceinline__ void qprime_sums_fp64(double qx, double q2, int p, double &S2m, double &S2, double &Qp1,
                                                 double &S)
{
    // U_{n-1}, U_n; S2m accumulates Q'_1..Q'_{p-1}.  The n = 1 step is
    // exact (U_2 = qx since gamma_1 = 0, S2m = lambda_1 U_1 = 1), so for p
    // >= 2 the loop starts at n = 2 (a product by U_0 = 0 would still cost
    // two multiplies and an add: IEEE arithmetic does not fold x * 0)
    double Um = 0.0, Uc = 1.0;
    S2m = 0.0;
    if (p >= 2) { Um = 1.0; Uc = qx; S2m = c_lambda<P>(1); }
    order_loop_up<P>(2, p, [&](int n) {
        S2m = fma(c_lambda<P>(n), Uc, S2m);
        const double Un = fma(qx, Uc, -(c_gamma<P>(n) * q2) * Um);
        Um = Uc; Uc = Un;
    });
    // Uc = U_p, Um = U_{p-1} (p >= 1);  p = 0: Q'_0 = 0, Q'_1 = 1
    double Qp = 0.0;
    Qp1 = 1.0;
    if (p >= 1) {
        Qp = c_lambda<P>(p) * Uc;
        Qp1 = c_lambda<P>(p + 1) * fma(qx, Uc, -(c_gamma<P>(p) * q2) * Um);
    }
    S2 = S2m + Qp;
    S = fma(fma(-2.0, qx, 1.0) + q2, S2, fma(-q2, Qp, Qp1));
}

template <int P, bool DLP, bool SP>
__device__ __forceinline__ void pair_fp64(double dx, double dy, double dz, double ex, double ey, double ez,
                                          double rho2, double wm, double nx, double ny, double nz,
                                          double tx, double ty, double tz, double ent,
                                          double &acc_s, double &acc_d, double &acc_p, int prt = 0)
{
    const int p = order_of<P>(prt);
    double rinv, r2inv, qx, q2;
    pair_geom_fp64(dx, dy, dz, ex, ey, ez, rho2, rinv, r2inv, qx, q2);
    const double wr = wm * rinv;
    if constexpr (!DLP && !SP) {
        acc_s = fma(wr, slp_clenshaw_fp64<P>(qx, q2, p), acc_s);
    } else {
        double S2m, S2, Qp1, S;
        qprime_sums_fp64<P>(qx, q2, p, S2m, S2, Qp1, S);
        acc_s = fma(wr, S, acc_s);
        const double wr3 = wr * r2inv;
        if (DLP) {
            const double a = fma(dx, nx, fma(dy, ny, dz * nz));
            const double b = fma(ex, nx, fma(ey, ny, ez * nz));
            acc_d = fma(wr3, fma(-a, Qp1, (b - a) * S2), acc_d);
        }
        if (SP) {
            const double dn = fma(dx, tx, fma(dy, ty, dz * tz));
            acc_p = fma(wr3, fma(dn, S2, -ent * S2m), acc_p);
        }
    }
}

// Write a target's sums (target j of the item): to the outputs, or to the
// partial-sum slots when the item is one slice of a longer list.
template <bool DLP, bool SP>
__device__ __forceinline__ void write_item_result(const DevGeom &g, const DevEval &ev, const Item &it, int j,
                                                  double acc_s, double acc_d, double acc_p)
{
    if (it.part < 0) {
        const int t = g.slot_tgt[it.slot_begin + j];
        if (ev.out_slp) ev.out_slp[t] = acc_s * kInv4Pi;
        if (DLP && ev.out_dlp) ev.out_dlp[t] = acc_d * kInv4Pi;
        if (SP && ev.out_sp) ev.out_sp[t] = acc_p * kInv4Pi;
    } else {
        if (ev.part_slp) ev.part_slp[it.part + j] = acc_s * kInv4Pi;
        if (DLP && ev.part_dlp) ev.part_dlp[it.part + j] = acc_d * kInv4Pi;
        if (SP && ev.part_sp) ev.part_sp[it.part + j] = acc_p * kInv4Pi;
    }
}

// Segmented sum over the L lanes of each target (lane sub == 0 gets it).
__device__ __forceinline__ double segment_sum(double v, int sub, int L)
{
    for (int off = 1; off < L; off <<= 1) {
        const double u = __shfl_down_sync(0xffffffffu, v, off);
        if (sub + off < L) v += u;
    }
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// T: the warp's staging tile, rows of `tile` doubles (x, y, z, w mu and, for
// the double layer, the normal's three components); tile is the staging depth
// (kTileMin..kTileMax sources per tile).
template <int P, bool DLP, bool SP>
__device__ __forceinline__ void laplace_fp64_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                  const WalkStart &ws, double *T, const int tile, const int lane)
{
    ListWalk walk(g, ws);
    const int src_hi = it.src_hi;
    double acc_s = 0.0, acc_d = 0.0, acc_p = 0.0;
    if (it.n_tgt == 1) {                                   // direct loads, all 32 lanes
        const double4_32a c = g.slot_c[it.slot_begin];
        const double4_32a e = g.slot_e[it.slot_begin];
        double tx = 0, ty = 0, tz = 0, ent = 0;
        if (SP) {
            const double4_32a tn = g.slot_n[it.slot_begin];
            tx = tn.x; ty = tn.y; tz = tn.z;
            ent = fma(e.x, tx, fma(e.y, ty, e.z * tz));                  // e.n_t
        }
#pragma unroll 2
        for (int k = it.src_lo + lane; k < src_hi; k += 32) {
            int s = walk.at(k);
            double wm = 0.0;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu[s];
            const double4_32a pw = g.src_pw[s];
            double nx = 0, ny = 0, nz = 0;
            if (DLP) { const double4_32a n = g.src_n[s]; nx = n.x; ny = n.y; nz = n.z; }
            pair_fp64<P, DLP, SP>(pw.x - c.x, pw.y - c.y, pw.z - c.z, e.x, e.y, e.z, e.w, wm, nx, ny, nz,
                                  tx, ty, tz, ent, acc_s, acc_d, acc_p, ev.p);
        }
        acc_s = warp_sum(acc_s);
        if (DLP) acc_d = warp_sum(acc_d);
        if (SP) acc_p = warp_sum(acc_p);
        if (lane == 0) write_item_result<DLP, SP>(g, ev, it, 0, acc_s, acc_d, acc_p);
        return;
    }
    const int L = it.L;
    const int j = lane / L, sub = lane - j * L;
    const bool active = j < it.n_tgt;
    double cx = 0, cy = 0, cz = 0, ex = 0, ey = 0, ez = 0, rho2 = 0, tx = 0, ty = 0, tz = 0, ent = 0;
    if (active) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double4_32a e = g.slot_e[it.slot_begin + j];
        cx = c.x; cy = c.y; cz = c.z;
        ex = e.x; ey = e.y; ez = e.z; rho2 = e.w;
        if (SP) {
            const double4_32a tn = g.slot_n[it.slot_begin + j];
            tx = tn.x; ty = tn.y; tz = tn.z;
            ent = fma(ex, tx, fma(ey, ty, ez * tz));                      // e.n_t
        }
    }
    double *const Tx = T, *const Ty = T + tile, *const Tz = T + 2 * tile, *const Tw = T + 3 * tile;
    double *const Nx = T + 4 * tile, *const Ny = T + 5 * tile, *const Nz = T + 6 * tile;   // DLP only
    for (int base = it.src_lo; base < src_hi; base += tile) {
        const int cnt = min(tile, src_hi - base);
        for (int k = lane; k < cnt; k += 32) {
            int s = walk.at(base + k);
            double wm = 0.0;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu[s];
            const double4_32a pw = g.src_pw[s];
            Tx[k] = pw.x; Ty[k] = pw.y; Tz[k] = pw.z; Tw[k] = wm;
            if (DLP) {
                const double4_32a n = g.src_n[s];
                Nx[k] = n.x; Ny[k] = n.y; Nz[k] = n.z;
            }
        }
        __syncwarp();
        if (active) {
            for (int k = sub; k < cnt; k += L)
                pair_fp64<P, DLP, SP>(Tx[k] - cx, Ty[k] - cy, Tz[k] - cz, ex, ey, ez, rho2, Tw[k],
                                      DLP ? Nx[k] : 0.0, DLP ? Ny[k] : 0.0, DLP ? Nz[k] : 0.0,
                                      tx, ty, tz, ent, acc_s, acc_d, acc_p, ev.p);
        }
        __syncwarp();
    }
    acc_s = segment_sum(acc_s, sub, L);
    if (DLP) acc_d = segment_sum(acc_d, sub, L);
    if (SP) acc_p = segment_sum(acc_p, sub, L);
    if (active && sub == 0) write_item_result<DLP, SP>(g, ev, it, j, acc_s, acc_d, acc_p);
}

// Several densities at once (DevEval::n_rhs = nr in 2..kMaxRhs): the
// per-pair kernel values -- S / R for the single layer, the double layer's
// bracket over R^3 -- depend on the geometry and the order alone, so the
// densities share them and each adds its own w mu with the same operations
// as pair_fp64 (wr = w mu / R, acc += wr S; DLP: wr3 = wr / R^2, acc_d +=
// wr3 val).  The double layer needs the normal n.
template <int P, bool DLP>
__device__ __forceinline__ void pair_fp64_multi(double dx, double dy, double dz, double ex, double ey, double ez,
                                                double rho2, double nx, double ny, double nz,
                                                const double (&wm)[kMaxRhs], double (&acc)[kMaxRhs],
                                                double (&acc_d)[kMaxRhs], int nr, int prt)
{
    const int p = order_of<P>(prt);
    double rinv, r2inv, qx, q2;
    pair_geom_fp64(dx, dy, dz, ex, ey, ez, rho2, rinv, r2inv, qx, q2);
    if constexpr (!DLP) {
        const double S = slp_clenshaw_fp64<P>(qx, q2, p);
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r)
            if (r < nr) acc[r] = fma(wm[r] * rinv, S, acc[r]);
    } else {
        double S2m, S2, Qp1, S;
        qprime_sums_fp64<P>(qx, q2, p, S2m, S2, Qp1, S);
        const double a = fma(dx, nx, fma(dy, ny, dz * nz));
        const double b = fma(ex, nx, fma(ey, ny, ez * nz));
        const double val = fma(-a, Qp1, (b - a) * S2);
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r)
            if (r < nr) {
                const double wr = wm[r] * rinv;
                acc[r] = fma(wr, S, acc[r]);
                acc_d[r] = fma(wr * r2inv, val, acc_d[r]);
            }
    }
}

// Result of density r for target j of an item: the single layer (DLP false)
// or the double layer of a multi-density evaluation, to its output or to its
// partial sums (part + r * rhs_part_stride) when the item is one slice.
template <bool DLP>
__device__ __forceinline__ void write_multi_result(const DevGeom &g, const DevEval &ev, const Item &it, int j, int r,
                                                   double acc)
{
    double *const out = DLP ? ev.out_rhs_dlp[r] : ev.out_rhs[r];
    double *const part = DLP ? ev.part_dlp : ev.part_slp;
    if (it.part < 0) {
        if (out) out[g.slot_tgt[it.slot_begin + j]] = acc * kInv4Pi;
    } else if (part) {
        part[r * ev.rhs_part_stride + it.part + j] = acc * kInv4Pi;
    }
}

// Staging rows of a multi-density item: x, y, z, (DLP) the normal's three
// components, then kMaxRhs rows of w mu.
__host__ __device__ constexpr int multi_tile_rows(bool dlp) { return (dlp ? 6 : 3) + kMaxRhs; }

// The single layer, and with DLP the double layer, for ev.n_rhs densities in
// one pass: the items, lanes, staging and reductions of laplace_fp64_item<P,
// DLP, false>, each density with its own accumulators, so that result r is
// bit-identical to the evaluation of density r alone.  T: multi_tile_rows(DLP)
// rows of `tile` doubles (density r's w mu in the row after the geometry's
// plus r).
template <int P, bool DLP>
__device__ __forceinline__ void laplace_fp64_multi_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                        const WalkStart &ws, double *T, const int tile,
                                                        const int lane)
{
    ListWalk walk(g, ws);
    const int src_hi = it.src_hi;
    const int nr = ev.n_rhs;
    const int64_t stride = ev.rhs_src_stride;
    double acc[kMaxRhs] = {0.0, 0.0, 0.0, 0.0}, acc_d[kMaxRhs] = {0.0, 0.0, 0.0, 0.0};
    if (it.n_tgt == 1) {                                   // direct loads, all 32 lanes
        const double4_32a c = g.slot_c[it.slot_begin];
        const double4_32a e = g.slot_e[it.slot_begin];
#pragma unroll 2
        for (int k = it.src_lo + lane; k < src_hi; k += 32) {
            int s = walk.at(k);
            const bool ok = (unsigned)s < (unsigned)g.n_src;
            if (!ok) { atomicOr(ev.status, 1); s = 0; }
            double wm[kMaxRhs];
#pragma unroll
            for (int r = 0; r < kMaxRhs; ++r) wm[r] = ok && r < nr ? ev.wmu[r * stride + s] : 0.0;
            const double4_32a pw = g.src_pw[s];
            double nx = 0, ny = 0, nz = 0;
            if (DLP) { const double4_32a n = g.src_n[s]; nx = n.x; ny = n.y; nz = n.z; }
            pair_fp64_multi<P, DLP>(pw.x - c.x, pw.y - c.y, pw.z - c.z, e.x, e.y, e.z, e.w, nx, ny, nz, wm, acc,
                                    acc_d, nr, ev.p);
        }
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r)
            if (r < nr) {
                const double v = warp_sum(acc[r]);
                const double vd = DLP ? warp_sum(acc_d[r]) : 0.0;
                if (lane == 0) {
                    write_multi_result<false>(g, ev, it, 0, r, v);
                    if (DLP) write_multi_result<true>(g, ev, it, 0, r, vd);
                }
            }
        return;
    }
    const int L = it.L;
    const int j = lane / L, sub = lane - j * L;
    const bool active = j < it.n_tgt;
    double cx = 0, cy = 0, cz = 0, ex = 0, ey = 0, ez = 0, rho2 = 0;
    if (active) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double4_32a e = g.slot_e[it.slot_begin + j];
        cx = c.x; cy = c.y; cz = c.z;
        ex = e.x; ey = e.y; ez = e.z; rho2 = e.w;
    }
    constexpr int kGeomRows = DLP ? 6 : 3;
    double *const Tx = T, *const Ty = T + tile, *const Tz = T + 2 * tile;
    double *const Nx = T + 3 * tile, *const Ny = T + 4 * tile, *const Nz = T + 5 * tile;   // DLP only
    double *const Tw = T + kGeomRows * tile;
    for (int base = it.src_lo; base < src_hi; base += tile) {
        const int cnt = min(tile, src_hi - base);
        for (int k = lane; k < cnt; k += 32) {
            int s = walk.at(base + k);
            const bool ok = (unsigned)s < (unsigned)g.n_src;
            if (!ok) { atomicOr(ev.status, 1); s = 0; }
            const double4_32a pw = g.src_pw[s];
            Tx[k] = pw.x; Ty[k] = pw.y; Tz[k] = pw.z;
            if (DLP) {
                const double4_32a n = g.src_n[s];
                Nx[k] = n.x; Ny[k] = n.y; Nz[k] = n.z;
            }
#pragma unroll
            for (int r = 0; r < kMaxRhs; ++r)
                if (r < nr) Tw[r * tile + k] = ok ? ev.wmu[r * stride + s] : 0.0;
        }
        __syncwarp();
        if (active) {
            for (int k = sub; k < cnt; k += L) {
                double wm[kMaxRhs];
#pragma unroll
                for (int r = 0; r < kMaxRhs; ++r) wm[r] = r < nr ? Tw[r * tile + k] : 0.0;
                pair_fp64_multi<P, DLP>(Tx[k] - cx, Ty[k] - cy, Tz[k] - cz, ex, ey, ez, rho2,
                                        DLP ? Nx[k] : 0.0, DLP ? Ny[k] : 0.0, DLP ? Nz[k] : 0.0, wm, acc, acc_d,
                                        nr, ev.p);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < kMaxRhs; ++r)
        if (r < nr) {
            const double v = segment_sum(acc[r], sub, L);
            const double vd = DLP ? segment_sum(acc_d[r], sub, L) : 0.0;
            if (active && sub == 0) {
                write_multi_result<false>(g, ev, it, j, r, v);
                if (DLP) write_multi_result<true>(g, ev, it, j, r, vd);
            }
        }
}

// Two (target, source) pairs at once in mixed precision, every FP32 operation
// packed (f32x2.cuh): the recurrences and closing sums of pair_fp64 in FP32,
// for the sources in the two halves, with s - c formed as (s_hi - c_hi) +
// (s_lo - c_lo) from float-float coordinates.  hx.. = source hi coordinates,
// w = w mu, lx.. = lo parts, mx.. = -n_s (the plan stores the source normals
// negated); ch/cl = center hi/lo, e = {t - c, -rho^2}, tn = {n_t, -e.n_t}
// (per target, both halves equal); one sum per layer, per half (KAHAN:
// compensated per pair; else a plain fused multiply-add, the caller
// compensating per tile).
//
// Operation count (p = 9, both layers, per pair): float-float difference 9,
// R^2 3, 1/R and 1/R^2 on the special-function unit, qx, -q2 and w/R 6,
// the Q' recurrence 4 per order from n = 2 (its n = 1 step is U_2 = qx,
// S2m = 1 exactly) and 3 at n = 2, its top 5, the closing sums 4, the double
// layer 11 with its sum, the single layer's sum 1.  Negated operands (-q2,
// -n_s, -e.n_t) are prepared outside the pair loop.

// Adds w * x to the packed sum s: Kahan-compensated (c the compensation) or
// a plain fused multiply-add.
template <bool KAHAN>
__device__ __forceinline__ void sum_fma2(f2 &s, f2 &c, f2 w, f2 x)
{
    if constexpr (KAHAN) kahan_add2(s, c, mul2(w, x));
    else s = fma2(w, x, s);
}

//
// MASK: a half whose flag (m0, m1) is set contributes an exact zero: its 1/R
// and 1/R^2 are taken as 0, so w/R, qx and q2 vanish and every term stays
// finite whatever the source's position (it may even sit on the center).
template <int P, bool DLP, bool SP, bool KAHAN = true, bool MASK = false>
__device__ __forceinline__ void pair_mixed2(f2 hx, f2 hy, f2 hz, f2 w, f2 lx, f2 ly, f2 lz, f2 mx, f2 my, f2 mz,
                                            const float4 &ch, const float4 &cl, const float4 &e,
                                            const float4 &tn, f2 &as, f2 &ac, f2 &ds, f2 &dc, f2 &ps, f2 &pc,
                                            bool m0 = false, bool m1 = false, int prt = 0)
{
    const int p = order_of<P>(prt);
    const f2 one = f2_splat(1.f);
    const f2 dx = add2(sub2(hx, f2_splat(ch.x)), sub2(lx, f2_splat(cl.x)));
    const f2 dy = add2(sub2(hy, f2_splat(ch.y)), sub2(ly, f2_splat(cl.y)));
    const f2 dz = add2(sub2(hz, f2_splat(ch.z)), sub2(lz, f2_splat(cl.z)));
    const f2 R2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    float r0, r1;
    f2_split(R2, r0, r1);
    float i0 = rsqrt_approx(r0), i1 = rsqrt_approx(r1);
    if constexpr (MASK) { i0 = m0 ? 0.f : i0; i1 = m1 ? 0.f : i1; }
    const f2 rinv = f2_make(i0, i1);
    // 1/R^2: rinv^2 for the single layer; with the double layer or S' its own
    // reciprocal (within 1 ulp): rinv's error (up to ~2 ulp) doubles in
    // rinv^2 and, through qx and q2, grows with the order in the Q'
    // recurrence
    f2 r2inv;
    if constexpr (DLP || SP) {
        float j0 = rcp_approx(r0), j1 = rcp_approx(r1);
        if constexpr (MASK) { j0 = m0 ? 0.f : j0; j1 = m1 ? 0.f : j1; }
        r2inv = f2_make(j0, j1);
    } else {
        r2inv = mul2(rinv, rinv);
    }
    const f2 qx = mul2(fma2(dx, f2_splat(e.x), fma2(dy, f2_splat(e.y), mul2(dz, f2_splat(e.z)))), r2inv);
    const f2 nq2 = mul2(f2_splat(e.w), r2inv);                       // -q2
    const f2 wr = mul2(w, rinv);
    if constexpr (!DLP && !SP) {
        // Clenshaw: b_k = kappa_k + qx b_{k+1} - beta_{k+1} q2 b_{k+2}
        f2 b1 = p >= 1 ? fma2(qx, f2_splat(c_kappa_f<P>(p)), f2_splat(c_kappa_f<P>(max(p - 1, 0)))) : one;
        f2 b2 = f2_splat(c_kappa_f<P>(p));
        order_loop_down<P>(0, p - 1, [&](int k) {
            const f2 bq = mul2(f2_splat(c_beta_f<P>(k + 1)), nq2);
            const f2 bk = fma2(bq, b2, fma2(qx, b1, f2_splat(c_kappa_f<P>(k))));
            b2 = b1; b1 = bk;
        });
        sum_fma2<KAHAN>(as, ac, wr, b1);
    } else {
        // U_{n-1}, U_n and S2m = sum_{m<n} Q'_m after the step of order n - 1:
        // at n = 2 (p >= 2) U_1 = 1, U_2 = qx (gamma_1 = 0), S2m = lambda_1 U_1 = 1
        f2 Um, Uc, S2m;
        if (p >= 2) { Um = one; Uc = qx; S2m = one; }
        else { Um = f2_splat(0.f); Uc = one; S2m = f2_splat(0.f); }
        if (p > 2) {                                   // n = 2, with U_1 = 1
            S2m = fma2(f2_splat(c_lambda_f<P>(2)), Uc, S2m);
            const f2 gq = mul2(f2_splat(c_gamma_f<P>(2)), nq2);
            const f2 Un = fma2(qx, Uc, gq);
            Um = Uc; Uc = Un;
        }
        order_loop_up<P>(3, p, [&](int n) {
            S2m = fma2(f2_splat(c_lambda_f<P>(n)), Uc, S2m);
            const f2 gq = mul2(f2_splat(c_gamma_f<P>(n)), nq2);          // -gamma_n q2
            const f2 Un = fma2(gq, Um, mul2(qx, Uc));
            Um = Uc; Uc = Un;
        });
        // Uc = U_p, Um = U_{p-1} (p >= 1);  p = 0: Q'_0 = 0, Q'_1 = 1
        f2 Qp = f2_splat(0.f), Qp1 = one;
        if (p >= 1) {
            Qp = mul2(f2_splat(c_lambda_f<P>(p)), Uc);
            const f2 gq = mul2(f2_splat(c_gamma_f<P>(p)), nq2);
            Qp1 = mul2(f2_splat(c_lambda_f<P>(p + 1)), fma2(gq, Um, mul2(qx, Uc)));
        }
        // S = (1 - 2 qx + q2) S2 + Q'_{p+1} - q2 Q'_p with S2 = S2m + Q'_p:
        //   = (1 - 2 qx + q2) S2m + (1 - 2 qx) Q'_p + Q'_{p+1}
        const f2 u = fma2(f2_splat(-2.f), qx, one);
        const f2 c1 = sub2(u, nq2);
        const f2 S = fma2(c1, S2m, fma2(u, Qp, Qp1));
        sum_fma2<KAHAN>(as, ac, wr, S);
        const f2 wr3 = mul2(wr, r2inv);
        const f2 S2 = add2(S2m, Qp);
        if (DLP) {
            // (b - a) S2 - a Q'_{p+1} with a = d.n_s, b = e.n_s, from the
            // negated normal: a' = -a, b' = -b give (a' - b') S2 + a' Q'_{p+1}
            const f2 am = fma2(dx, mx, fma2(dy, my, mul2(dz, mz)));
            const f2 bm = fma2(f2_splat(e.x), mx, fma2(f2_splat(e.y), my, mul2(f2_splat(e.z), mz)));
            sum_fma2<KAHAN>(ds, dc, wr3, fma2(am, Qp1, mul2(sub2(am, bm), S2)));
        }
        if (SP) {
            // (d.n_t) S2 - (e.n_t) S2m, tn.w = -e.n_t
            const f2 dn = fma2(dx, f2_splat(tn.x), fma2(dy, f2_splat(tn.y), mul2(dz, f2_splat(tn.z))));
            sum_fma2<KAHAN>(ps, pc, wr3, fma2(dn, S2, mul2(f2_splat(tn.w), S2m)));
        }
    }
}

// A lane's Kahan-compensated packed sums (two halves, each s - c) as one
// double-float value, and its sums across lanes in double-float: the lanes'
// partial sums meet on the FP32 pipes, and only the writing lane converts the
// total to FP64.  (An FP64 reduction per item costs ~12 FP64 operations per
// lane, which on a 2-DFMA/clk/SM part rivals the pair work of short lists.)
__device__ __forceinline__ df kahan2_df(f2 s, f2 c)
{
    float s0, s1, c0, c1;
    f2_split(s, s0, s1);
    f2_split(c, c0, c1);
    return df_add(two_sum(s0, -c0), two_sum(s1, -c1));
}

__device__ __forceinline__ df df_shfl_xor(df v, int off)
{
    return df{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}

__device__ __forceinline__ df warp_sum_df(df v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = df_add(v, df_shfl_xor(v, off));
    return v;
}

// Sum over the L lanes of each target's segment (sub = 0 holds the total);
// a target's lanes are `stride` apart (lane = sub * stride + target).
__device__ __forceinline__ df segment_sum_df(df v, int sub, int L, int stride = 1)
{
    for (int off = 1; off < L; off <<= 1) {
        const df u{__shfl_down_sync(0xffffffffu, v.hi, off * stride),
                   __shfl_down_sync(0xffffffffu, v.lo, off * stride)};
        if (sub + off < L) v = df_add(v, u);
    }
    return v;
}

// Shared-memory tile of the mixed item, two sources per record (record j
// holds sources 2j and 2j+1 of the tile) of five 16-byte words: {hx0, hx1,
// hy0, hy1}, {hz0, hz1, w0, w1}, {lx0, lx1, ly0, ly1}, {lz0, lz1, mx0, mx1}
// and, for the double layer, {my0, my1, mz0, mz1} (m = -n_s; unused by the
// single layer).  One 16-byte load gives two packed operands; the records of
// a tile are consecutive, so one address and constant offsets reach a
// record's words, and their odd length (80 bytes) puts the records that
// eight lanes read at once on distinct banks.  tile / 2 records per tile.
__host__ __device__ constexpr int mixed_tile_rows(bool) { return 5; }
// Longest run of source pairs a lane sums in plain FP32 before adding the run
// to its compensated sums: the rounding error of a plain run grows with its
// length, so deeper tiles do not lengthen it.
constexpr int kPlainRun = 16;

// Load the list positions k0 and k1 (k1 < 0: a zero-weight copy of k0) of a
// group's list as packed operands; k0 < k1, neither before the walk's last call.
template <bool DLP>
__device__ __forceinline__ void load_mixed_pair(const DevGeom &g, const DevEval &ev, ListWalk &walk, int k0, int k1,
                                                f2 &hx, f2 &hy, f2 &hz, f2 &w, f2 &lx, f2 &ly, f2 &lz, f2 &nx,
                                                f2 &ny, f2 &nz)
{
    int sa = walk.at(k0);
    int sb = k1 >= 0 ? walk.at(k1) : sa;
    float wa = 0.f, wb = 0.f;
    if ((unsigned)sa >= (unsigned)g.n_src) { atomicOr(ev.status, 1); sa = 0; } else wa = ev.wmu_f[sa];
    if ((unsigned)sb >= (unsigned)g.n_src) { atomicOr(ev.status, 1); sb = 0; } else if (k1 >= 0) wb = ev.wmu_f[sb];
    const float4 ha = g.src_hi[sa], hb = g.src_hi[sb], la = g.src_lo[sa], lb = g.src_lo[sb];
    hx = f2_make(ha.x, hb.x); hy = f2_make(ha.y, hb.y); hz = f2_make(ha.z, hb.z); w = f2_make(wa, wb);
    lx = f2_make(la.x, lb.x); ly = f2_make(la.y, lb.y); lz = f2_make(la.z, lb.z);
    if (DLP) {
        const float4 na = g.src_nf[sa], nb = g.src_nf[sb];
        nx = f2_make(na.x, nb.x); ny = f2_make(na.y, nb.y); nz = f2_make(na.z, nb.z);
    } else {
        nx = ny = nz = f2_splat(0.f);
    }
}

// A single-target item of the single layer on W lanes of a warp (W = 16 or
// 8; sl = lane within the group), so that a warp works 32/W such items at
// once and their dependent loads overlap: each lane takes sources k and k + W
// of every 2W, and the group reduces over its W lanes (xor offsets below W
// stay within a group).  Every group must run the same P.
template <int P, int W>
__device__ __forceinline__ void laplace_mixed_part_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                        const WalkStart &ws, const int sl)
{
    ListWalk walk(g, ws);
    const int src_hi = it.src_hi;
    const f2 z2 = f2_splat(0.f);
    f2 as = z2, ac = z2, unused = z2;
    const float4 ch = g.slot_chi[it.slot_begin];
    const float4 cl = g.slot_clo[it.slot_begin];
    const float4 e = g.slot_ef[it.slot_begin];
    const float4 tn = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = it.src_lo + sl; k < src_hi; k += 2 * W) {
        f2 hx, hy, hz, w, lx, ly, lz, nx, ny, nz;
        load_mixed_pair<false>(g, ev, walk, k, k + W < src_hi ? k + W : -1, hx, hy, hz, w, lx, ly, lz, nx, ny, nz);
        pair_mixed2<P, false, false>(hx, hy, hz, w, lx, ly, lz, nx, ny, nz, ch, cl, e, tn, as, ac, unused, unused,
                                     unused, unused);
    }
    df v = kahan2_df(as, ac);
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v = df_add(v, df_shfl_xor(v, off));
    if (sl == 0) write_item_result<false, false>(g, ev, it, 0, df_to_double(v), 0.0, 0.0);
}

// The source range [a, b) of a single-target item whose slice lies in one run
// of its group's list (the run's sources are consecutive); false otherwise.
__device__ __forceinline__ bool single_run_range(const Item &it, const WalkStart &ws, int32_t &a, int32_t &b)
{
    if (it.n_tgt != 1 || it.src_hi > ws.p1 || it.src_lo < ws.p0) return false;
    a = ws.s0 + (it.src_lo - ws.p0);
    b = ws.s0 + (it.src_hi - ws.p0);
    return true;
}

// Four single-target items of one single-layer mixed plan whose sources are
// the consecutive ranges [a_q, b_q) (one run each), read through their union
// [A, B): the warp stages the union in tiles of kTile sources (the pair
// records of the mixed tile) and each item's 8 lanes (q = lane % 4, sl = lane
// / 4) take, in step with the other items' lanes, every record of the tile,
// a record half outside the item's range masked to an exact zero (its 1/R
// taken as 0).  Neighbouring centers of a
// surface list overlapping windows, so the union is little longer than each:
// one load of a source record serves every item that lists it.  Plain FP32
// sums per tile, Kahan across tiles, double-float across the 8 lanes.
template <int P>
__device__ __forceinline__ void laplace_mixed_window4(const DevGeom &g, const DevEval &ev, const Item &it,
                                                      int32_t a, int32_t b, int32_t A, int32_t B, float4 *T,
                                                      const int lane)
{
    constexpr int kPairs = kTile / 2;
    float4 *const T0 = T, *const T1 = T + kPairs, *const T2 = T + 2 * kPairs, *const T3 = T + 3 * kPairs;
    const int sl = lane >> 2;
    const f2 z2 = f2_splat(0.f);
    f2 as = z2, ac = z2, unused = z2;
    const float4 ch = g.slot_chi[it.slot_begin];
    const float4 cl = g.slot_clo[it.slot_begin];
    const float4 e = g.slot_ef[it.slot_begin];
    const float4 tn = make_float4(0.f, 0.f, 0.f, 0.f);
    // record `lane` of a tile holds sources base + lane and base + lane +
    // kPairs, so that the warp's loads of each array are contiguous.  The
    // loads of the next tile are issued before the current tile's sums and
    // stored after them, so their latency overlaps the arithmetic.
    float4 h0, h1, l0, l1;
    float w0, w1;
    auto fetch = [&](int32_t base) {
        int32_t s0 = base + lane, s1 = s0 + kPairs;
        w0 = 0.f; w1 = 0.f;
        if (s0 < B && (unsigned)s0 < (unsigned)g.n_src) w0 = ev.wmu_f[s0];
        else s0 = 0;
        if (s1 < B && (unsigned)s1 < (unsigned)g.n_src) w1 = ev.wmu_f[s1];
        else s1 = s0;
        h0 = g.src_hi[s0]; h1 = g.src_hi[s1]; l0 = g.src_lo[s0]; l1 = g.src_lo[s1];
    };
    fetch(A);
    for (int32_t base = A; base < B; base += kTile) {
        T0[lane] = make_float4(h0.x, h1.x, h0.y, h1.y);
        T1[lane] = make_float4(h0.z, h1.z, w0, w1);
        T2[lane] = make_float4(l0.x, l1.x, l0.y, l1.y);
        T3[lane] = make_float4(l0.z, l1.z, 0.f, 0.f);
        __syncwarp();
        if (base + kTile < B) fetch(base + kTile);
        // the four items walk the tile's records in step (lane sl of every item
        // reads the same record, and the four such lanes sit in one
        // quarter-warp: one shared-memory broadcast serves four), each
        // taking the halves that fall in its own sources max(a, base) ..
        // min(b, base + kTile) - 1; a half outside them (another item's source,
        // which this center does not list and may even coincide with) is
        // masked to an exact zero, without a branch
        const int32_t lo = max(a, base) - base, n_in = max(min(b, base + kTile) - base - lo, 0);
        f2 ts = z2;
#pragma unroll
        for (int k = 0; k < kPairs / 8; ++k) {
            const int i = sl + 8 * k;
            const bool m0 = (unsigned)(i - lo) >= (unsigned)n_in, m1 = (unsigned)(i + kPairs - lo) >= (unsigned)n_in;
            const float4 A4 = T0[i], B4 = T1[i], C4 = T2[i], D4 = T3[i];
            pair_mixed2<P, false, false, false, true>(f2_xy(A4), f2_zw(A4), f2_xy(B4), f2_zw(B4), f2_xy(C4),
                                                      f2_zw(C4), f2_xy(D4), z2, z2, z2, ch, cl, e, tn, ts, unused,
                                                      unused, unused, unused, unused, m0, m1);
        }
        kahan_add2(as, ac, ts);
        __syncwarp();
    }
    df v = kahan2_df(as, ac);
#pragma unroll
    for (int off = 16; off >= 4; off >>= 1) v = df_add(v, df_shfl_xor(v, off));   // sl ^ 4, ^ 2, ^ 1
    if (sl == 0) write_item_result<false, false>(g, ev, it, 0, df_to_double(v), 0.0, 0.0);
}

template <int P, bool DLP, bool SP>
__device__ __forceinline__ void laplace_mixed_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                   const WalkStart &ws, float4 *T, const int tile, const int lane)
{
    ListWalk walk(g, ws);
    const int src_hi = it.src_hi;
    const f2 z2 = f2_splat(0.f);
    f2 as = z2, ac = z2, ds = z2, dc = z2, ps = z2, pc = z2;   // Kahan pairs
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    if (it.n_tgt == 1) {                               // direct loads, all 32 lanes, two sources each
        const float4 ch = g.slot_chi[it.slot_begin];
        const float4 cl = g.slot_clo[it.slot_begin];
        const float4 e = g.slot_ef[it.slot_begin];
        const float4 tn = SP ? g.slot_nf[it.slot_begin] : zero;
        for (int k = it.src_lo + lane; k < src_hi; k += 64) {
            f2 hx, hy, hz, w, lx, ly, lz, nx, ny, nz;
            load_mixed_pair<DLP>(g, ev, walk, k, k + 32 < src_hi ? k + 32 : -1, hx, hy, hz, w, lx, ly, lz, nx, ny, nz);
            pair_mixed2<P, DLP, SP>(hx, hy, hz, w, lx, ly, lz, nx, ny, nz, ch, cl, e, tn, as, ac, ds, dc, ps, pc,
                                    false, false, ev.p);
        }
        const df acc_s = warp_sum_df(kahan2_df(as, ac));
        const df acc_d = DLP ? warp_sum_df(kahan2_df(ds, dc)) : df{0.f, 0.f};
        const df acc_p = SP ? warp_sum_df(kahan2_df(ps, pc)) : df{0.f, 0.f};
        if (lane == 0)
            write_item_result<DLP, SP>(g, ev, it, 0, df_to_double(acc_s), df_to_double(acc_d), df_to_double(acc_p));
        return;
    }
    // target j = lane % n_tgt, its L lanes n_tgt apart: the lanes of the
    // item's targets that read one staged record sit together, so that a
    // shared-memory load serves them in fewer wavefronts
    const int L = it.L, nt = it.n_tgt;
    const int sub = lane / nt, j = lane - sub * nt;
    const bool active = sub < L;
    float4 ch = zero, cl = zero, e = zero, tn = zero;
    if (active) {
        ch = g.slot_chi[it.slot_begin + j];
        cl = g.slot_clo[it.slot_begin + j];
        e = g.slot_ef[it.slot_begin + j];
        if (SP) tn = g.slot_nf[it.slot_begin + j];
    }
    constexpr int kRec = mixed_tile_rows(DLP);         // 16-byte words per record
    for (int base = it.src_lo; base < src_hi; base += tile) {
        const int cnt = min(tile, src_hi - base);
        const int npairs = (cnt + 1) >> 1;
        for (int q = lane; q < npairs; q += 32) {      // lane stages pairs lane, lane + 32, ...
            const int k0 = base + 2 * q;
            f2 hx, hy, hz, w, lx, ly, lz, nx, ny, nz;
            load_mixed_pair<DLP>(g, ev, walk, k0, 2 * q + 1 < cnt ? k0 + 1 : -1, hx, hy, hz, w, lx, ly, lz, nx,
                                 ny, nz);
            float a0, a1, b0, b1;
            float4 *const r = T + q * kRec;
            f2_split(hx, a0, a1); f2_split(hy, b0, b1); r[0] = make_float4(a0, a1, b0, b1);
            f2_split(hz, a0, a1); f2_split(w, b0, b1);  r[1] = make_float4(a0, a1, b0, b1);
            f2_split(lx, a0, a1); f2_split(ly, b0, b1); r[2] = make_float4(a0, a1, b0, b1);
            f2_split(lz, a0, a1); f2_split(nx, b0, b1); r[3] = make_float4(a0, a1, b0, b1);
            if (DLP) { f2_split(ny, a0, a1); f2_split(nz, b0, b1); r[4] = make_float4(a0, a1, b0, b1); }
        }
        __syncwarp();
        if (active) {
            // plain FP32 sums over runs of at most kPlainRun source pairs per
            // lane, each run added to the compensated sums (at the default
            // depth and L >= 2, one run per tile)
            for (int q0 = sub; q0 < npairs; q0 += kPlainRun * L) {
                const int q1 = min(npairs, q0 + kPlainRun * L);
                f2 ts = z2, td = z2, tp2 = z2, unused = z2;
                for (int q = q0; q < q1; q += L) {
                    const float4 *const r = T + q * kRec;
                    const float4 A = r[0], B = r[1], C = r[2], D = r[3];
                    const float4 E = DLP ? r[4] : zero;
                    pair_mixed2<P, DLP, SP, false>(f2_xy(A), f2_zw(A), f2_xy(B), f2_zw(B), f2_xy(C), f2_zw(C),
                                                   f2_xy(D), f2_zw(D), f2_xy(E), f2_zw(E), ch, cl, e, tn, ts,
                                                   unused, td, unused, tp2, unused, false, false, ev.p);
                }
                kahan_add2(as, ac, ts);
                if (DLP) kahan_add2(ds, dc, td);
                if (SP) kahan_add2(ps, pc, tp2);
            }
        }
        __syncwarp();
    }
    const df acc_s = segment_sum_df(kahan2_df(as, ac), sub, L, nt);
    const df acc_d = DLP ? segment_sum_df(kahan2_df(ds, dc), sub, L, nt) : df{0.f, 0.f};
    const df acc_p = SP ? segment_sum_df(kahan2_df(ps, pc), sub, L, nt) : df{0.f, 0.f};
    if (active && sub == 0)
        write_item_result<DLP, SP>(g, ev, it, j, df_to_double(acc_s), df_to_double(acc_d), df_to_double(acc_p));
}

}  // namespace tsqbx
