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

#include "internal.cuh"

namespace tsqbx {

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

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
//   double layer  n_s.grad_s (S/R) = (1/R^3) [ -a S1 + (b - a qx) S2 ],
//   S'            n_t.grad_t (S/R) = (1/R^3) [ (d.n_t) S2 - (e.n_t) S2m ],
// a = d.n_s, b = e.n_s.  The closing sums cancel at most by a factor of a few
// hundred over rho/R <= 0.9, orders 0..20, a cost of ~2e-14 in FP64.
template <int P, bool DLP, bool SP>
__device__ __forceinline__ void pair_fp64(double dx, double dy, double dz, double ex, double ey, double ez,
                                          double rho2, double wm, double nx, double ny, double nz,
                                          double tx, double ty, double tz, double ent,
                                          double &acc_s, double &acc_d, double &acc_p)
{
    const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double rinv = rsqrt(R2);
    const double r2inv = rinv * rinv;
    const double qx = fma(dx, ex, fma(dy, ey, dz * ez)) * r2inv;
    const double q2 = rho2 * r2inv;
    const double wr = wm * rinv;
    if constexpr (!DLP && !SP) {
        // b_{k+1}, b_{k+2} at k = P - 2 (b_{P+1} = 0 drops out of b_{P-1})
        double b1 = P >= 1 ? fma(qx, rec_kappa(P), rec_kappa(P - 1)) : 1.0, b2 = rec_kappa(P);
#pragma unroll
        for (int k = P - 2; k >= 0; --k) {
            const double bk = fma(-(rec_beta(k + 1) * q2), b2, fma(qx, b1, rec_kappa(k)));
            b2 = b1; b1 = bk;
        }
        acc_s = fma(wr, b1, acc_s);
    } else {
        // U_{n-1}, U_n starting at n = 1; S2m accumulates Q'_1..Q'_{P-1}
        double Um = 0.0, Uc = 1.0, S2m = 0.0;
#pragma unroll
        for (int n = 1; n < P; ++n) {
            S2m = fma(rec_lambda(n), Uc, S2m);
            const double Un = fma(qx, Uc, -(rec_gamma(n) * q2) * Um);
            Um = Uc; Uc = Un;
        }
        // Uc = U_P, Um = U_{P-1} (P >= 1);  P = 0: Q'_0 = 0, Q'_1 = 1
        const double Qp = P >= 1 ? rec_lambda(P) * Uc : 0.0;
        const double Qp1 = P >= 1 ? rec_lambda(P + 1) * fma(qx, Uc, -(rec_gamma(P) * q2) * Um) : 1.0;
        const double S2 = S2m + Qp;
        const double S = fma(fma(-2.0, qx, 1.0) + q2, S2, fma(-q2, Qp, Qp1));
        acc_s = fma(wr, S, acc_s);
        const double wr3 = wr * r2inv;
        if (DLP) {
            const double S1 = fma(1.0 - qx, S2, Qp1);
            const double a = fma(dx, nx, fma(dy, ny, dz * nz));
            const double b = fma(ex, nx, fma(ey, ny, ez * nz));
            acc_d = fma(wr3, fma(-a, S1, fma(-a, qx, b) * S2), acc_d);
        }
        if (SP) {
            const double dn = fma(dx, tx, fma(dy, ty, dz * tz));
            acc_p = fma(wr3, fma(dn, S2, -ent * S2m), acc_p);
        }
    }
}

// One pair in mixed precision: h/l = source hi/lo (h.w = w mu), ch/cl = center
// hi/lo, e = {t - c, rho^2}, nn = n_s, tn = {n_t, e.n_t}; Kahan-compensated
// FP32 sums (as/ac single layer, ds/dc double layer, ps/pc S').  Same two
// recurrences and closing sums as pair_fp64, in FP32.
template <int P, bool DLP, bool SP>
__device__ __forceinline__ void pair_mixed(const float4 &h, const float4 &l, const float4 &ch, const float4 &cl,
                                           const float4 &e, const float4 &nn, const float4 &tn, float &as,
                                           float &ac, float &ds, float &dc, float &ps, float &pc)
{
    const float dx = __fadd_rn(__fsub_rn(h.x, ch.x), __fsub_rn(l.x, cl.x));
    const float dy = __fadd_rn(__fsub_rn(h.y, ch.y), __fsub_rn(l.y, cl.y));
    const float dz = __fadd_rn(__fsub_rn(h.z, ch.z), __fsub_rn(l.z, cl.z));
    const float R2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = rsqrtf(R2);
    const float r2inv = rinv * rinv;
    const float qx = fmaf(dx, e.x, fmaf(dy, e.y, dz * e.z)) * r2inv;
    const float q2 = e.w * r2inv;
    const float wr = h.w * rinv;
    if constexpr (!DLP && !SP) {
        float b1 = P >= 1 ? fmaf(qx, (float)rec_kappa(P), (float)rec_kappa(P - 1)) : 1.f;   // as pair_fp64
        float b2 = (float)rec_kappa(P);
#pragma unroll
        for (int k = P - 2; k >= 0; --k) {
            const float bk = fmaf(-((float)rec_beta(k + 1) * q2), b2, fmaf(qx, b1, (float)rec_kappa(k)));
            b2 = b1; b1 = bk;
        }
        kahan_add(as, ac, wr * b1);
    } else {
        float Um = 0.f, Uc = 1.f, S2m = 0.f;
#pragma unroll
        for (int n = 1; n < P; ++n) {
            S2m = fmaf((float)rec_lambda(n), Uc, S2m);
            const float Un = fmaf(qx, Uc, -((float)rec_gamma(n) * q2) * Um);
            Um = Uc; Uc = Un;
        }
        const float Qp = P >= 1 ? (float)rec_lambda(P) * Uc : 0.f;
        const float Qp1 = P >= 1 ? (float)rec_lambda(P + 1) * fmaf(qx, Uc, -((float)rec_gamma(P) * q2) * Um) : 1.f;
        const float S2 = S2m + Qp;
        const float S = fmaf(fmaf(-2.f, qx, 1.f) + q2, S2, fmaf(-q2, Qp, Qp1));
        kahan_add(as, ac, wr * S);
        const float wr3 = wr * r2inv;
        if (DLP) {
            const float S1 = fmaf(1.f - qx, S2, Qp1);
            const float a = fmaf(dx, nn.x, fmaf(dy, nn.y, dz * nn.z));
            const float b = fmaf(e.x, nn.x, fmaf(e.y, nn.y, e.z * nn.z));
            kahan_add(ds, dc, wr3 * fmaf(-a, S1, fmaf(-a, qx, b) * S2));
        }
        if (SP) {
            const float dn = fmaf(dx, tn.x, fmaf(dy, tn.y, dz * tn.z));
            kahan_add(ps, pc, wr3 * fmaf(dn, S2, -tn.w * S2m));
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

template <int P, bool DLP, bool SP>
__device__ __forceinline__ void laplace_fp64_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                  double (*T)[kTile], const int lane)
{
    const int64_t s0 = g.grp_off[it.group];
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
            int s = g.grp_src[s0 + k];
            double wm = 0.0;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu[s];
            const double4_32a pw = g.src_pw[s];
            double nx = 0, ny = 0, nz = 0;
            if (DLP) { const double4_32a n = g.src_n[s]; nx = n.x; ny = n.y; nz = n.z; }
            pair_fp64<P, DLP, SP>(pw.x - c.x, pw.y - c.y, pw.z - c.z, e.x, e.y, e.z, e.w, wm, nx, ny, nz,
                                  tx, ty, tz, ent, acc_s, acc_d, acc_p);
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
    for (int base = it.src_lo; base < src_hi; base += kTile) {
        const int cnt = min(kTile, src_hi - base);
        for (int k = lane; k < cnt; k += 32) {
            int s = g.grp_src[s0 + base + k];
            double wm = 0.0;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu[s];
            const double4_32a pw = g.src_pw[s];
            T[0][k] = pw.x; T[1][k] = pw.y; T[2][k] = pw.z; T[3][k] = wm;
            if (DLP) {
                const double4_32a n = g.src_n[s];
                T[4][k] = n.x; T[5][k] = n.y; T[6][k] = n.z;
            }
        }
        __syncwarp();
        if (active) {
            for (int k = sub; k < cnt; k += L)
                pair_fp64<P, DLP, SP>(T[0][k] - cx, T[1][k] - cy, T[2][k] - cz, ex, ey, ez, rho2, T[3][k],
                                      DLP ? T[4][k] : 0.0, DLP ? T[5][k] : 0.0, DLP ? T[6][k] : 0.0,
                                      tx, ty, tz, ent, acc_s, acc_d, acc_p);
        }
        __syncwarp();
    }
    acc_s = segment_sum(acc_s, sub, L);
    if (DLP) acc_d = segment_sum(acc_d, sub, L);
    if (SP) acc_p = segment_sum(acc_p, sub, L);
    if (active && sub == 0) write_item_result<DLP, SP>(g, ev, it, j, acc_s, acc_d, acc_p);
}

template <int P, bool DLP, bool SP>
__device__ __forceinline__ void laplace_mixed_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                   float4 (*T)[kTile], const int lane)
{
    const int64_t s0 = g.grp_off[it.group];
    const int src_hi = it.src_hi;
    float as = 0.f, ac = 0.f, ds = 0.f, dc = 0.f, ps = 0.f, pc = 0.f;   // Kahan pairs
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    if (it.n_tgt == 1) {                               // direct loads, all 32 lanes
        const float4 ch = g.slot_chi[it.slot_begin];
        const float4 cl = g.slot_clo[it.slot_begin];
        const float4 e = g.slot_ef[it.slot_begin];
        float4 tn = zero;
        if (SP) {
            tn = g.slot_nf[it.slot_begin];
            tn.w = fmaf(e.x, tn.x, fmaf(e.y, tn.y, e.z * tn.z));    // e.n_t
        }
#pragma unroll 2
        for (int k = it.src_lo + lane; k < src_hi; k += 32) {
            int s = g.grp_src[s0 + k];
            float wm = 0.f;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu_f[s];
            float4 h = g.src_hi[s];
            h.w = wm;
            const float4 l = g.src_lo[s];
            const float4 nn = DLP ? g.src_nf[s] : zero;
            pair_mixed<P, DLP, SP>(h, l, ch, cl, e, nn, tn, as, ac, ds, dc, ps, pc);
        }
        const double acc_s = warp_sum((double)as - (double)ac);
        const double acc_d = DLP ? warp_sum((double)ds - (double)dc) : 0.0;
        const double acc_p = SP ? warp_sum((double)ps - (double)pc) : 0.0;
        if (lane == 0) write_item_result<DLP, SP>(g, ev, it, 0, acc_s, acc_d, acc_p);
        return;
    }
    const int L = it.L;
    const int j = lane / L, sub = lane - j * L;
    const bool active = j < it.n_tgt;
    float4 ch = zero, cl = zero, e = zero, tn = zero;
    if (active) {
        ch = g.slot_chi[it.slot_begin + j];
        cl = g.slot_clo[it.slot_begin + j];
        e = g.slot_ef[it.slot_begin + j];
        if (SP) {
            tn = g.slot_nf[it.slot_begin + j];
            tn.w = fmaf(e.x, tn.x, fmaf(e.y, tn.y, e.z * tn.z));    // e.n_t
        }
    }
    for (int base = it.src_lo; base < src_hi; base += kTile) {
        const int cnt = min(kTile, src_hi - base);
        for (int k = lane; k < cnt; k += 32) {
            int s = g.grp_src[s0 + base + k];
            float wm = 0.f;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wm = ev.wmu_f[s];
            float4 h = g.src_hi[s];
            h.w = wm;
            T[0][k] = h;
            T[1][k] = g.src_lo[s];
            if (DLP) T[2][k] = g.src_nf[s];
        }
        __syncwarp();
        if (active) {
            for (int k = sub; k < cnt; k += L)
                pair_mixed<P, DLP, SP>(T[0][k], T[1][k], ch, cl, e, DLP ? T[2][k] : zero, tn, as, ac, ds, dc,
                                       ps, pc);
        }
        __syncwarp();
    }
    const double acc_s = segment_sum((double)as - (double)ac, sub, L);
    const double acc_d = DLP ? segment_sum((double)ds - (double)dc, sub, L) : 0.0;
    const double acc_p = SP ? segment_sum((double)ps - (double)pc, sub, L) : 0.0;
    if (active && sub == 0) write_item_result<DLP, SP>(g, ev, it, j, acc_s, acc_d, acc_p);
}

}  // namespace tsqbx
