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

// One (target, source) pair in FP64: d = s - c, e = t - c, wm = w mu, n = n_s.
// S' (target-normal derivative): the recurrence differentiated along n_t,
// T'_{n+1} = qx' T_n + qx T'_n - beta_n (q2' T_{n-1} + q2 T'_{n-1}) with
// qx' = (d.n_t)/R^2 and q2' = 2 (e.n_t)/R^2 (f2 = 2 e.n_t, per target), so
// n_t.grad_t G^(p) = (1/4pi)(1/R) sum kappa_n T'_n -- no division by rho.
template <int P, bool DLP, bool SP>
__device__ __forceinline__ void pair_fp64(double dx, double dy, double dz, double ex, double ey, double ez,
                                          double rho2, double wm, double nx, double ny, double nz,
                                          double tx, double ty, double tz, double f2,
                                          double &acc_s, double &acc_d, double &acc_p)
{
    const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double rinv = rsqrt(R2);
    const double r2inv = rinv * rinv;
    const double qx = fma(dx, ex, fma(dy, ey, dz * ez)) * r2inv;
    const double q2 = rho2 * r2inv;
    const double qxp = SP ? fma(dx, tx, fma(dy, ty, dz * tz)) * r2inv : 0.0;
    const double q2p = SP ? f2 * r2inv : 0.0;
    // n = 0 (and n = 1 when P >= 1); T_{n-1}, T_n, Q'_{n-1}, Q'_n, T'_{n-1}, T'_n
    double S0 = 1.0, S2 = 0.0, S3 = 0.0;
    double Tm = 1.0, Tc = 1.0, Dm = 0.0, Dc = 0.0, Pm = 0.0, Pc = 0.0;
    if (P >= 1) { S0 += qx; S2 = 1.0; Tc = qx; Dc = 1.0; Pc = qxp; S3 = qxp; }
#pragma unroll
    for (int n = 1; n < P; ++n) {
        const double Tn = fma(qx, Tc, -(rec_beta(n) * q2) * Tm);
        S0 = fma(rec_kappa(n + 1), Tn, S0);
        if (DLP) {
            const double Dn = fma(q2, Dm, ((2.0 * n + 1.0) * rec_kappa(n)) * Tc);
            S2 += Dn;
            Dm = Dc; Dc = Dn;
        }
        if (SP) {
            const double Pn = fma(qxp, Tc, fma(qx, Pc, -rec_beta(n) * fma(q2p, Tm, q2 * Pm)));
            S3 = fma(rec_kappa(n + 1), Pn, S3);
            Pm = Pc; Pc = Pn;
        }
        Tm = Tc; Tc = Tn;
    }
    acc_s = fma(wm * rinv, S0, acc_s);
    if (SP) acc_p = fma(wm * rinv, S3, acc_p);
    if (DLP) {
        const double Dp1 = fma(q2, Dm, ((2.0 * P + 1.0) * rec_kappa(P)) * Tc);
        const double S1 = 0.5 * (fma(-q2, S2, S2) + Dp1 + fma(q2, Dc, S0));
        const double a = fma(dx, nx, fma(dy, ny, dz * nz));
        const double b = fma(ex, nx, fma(ey, ny, ez * nz));
        const double val = fma(-a, S1, fma(-a, qx, b) * S2);
        acc_d = fma(wm * rinv * r2inv, val, acc_d);
    }
}

// One pair in mixed precision: h/l = source hi/lo (h.w = w mu), ch/cl = center
// hi/lo, e = {t - c, rho^2}, nn = n_s, tn = {n_t, 2 e.n_t}; Kahan-compensated
// FP32 sums (as/ac single layer, ds/dc double layer, ps/pc S').
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
    const float qxp = SP ? fmaf(dx, tn.x, fmaf(dy, tn.y, dz * tn.z)) * r2inv : 0.f;
    const float q2p = SP ? tn.w * r2inv : 0.f;
    float S0 = 1.f, S2 = 0.f, S3 = 0.f;
    float Tm = 1.f, Tc = 1.f, Dm = 0.f, Dc = 0.f, Pm = 0.f, Pc = 0.f;
    if (P >= 1) { S0 += qx; S2 = 1.f; Tc = qx; Dc = 1.f; Pc = qxp; S3 = qxp; }
#pragma unroll
    for (int n = 1; n < P; ++n) {
        const float Tn = fmaf(qx, Tc, -((float)rec_beta(n) * q2) * Tm);
        S0 = fmaf((float)rec_kappa(n + 1), Tn, S0);
        if (DLP) {
            const float Dn = fmaf(q2, Dm, (float)((2.0 * n + 1.0) * rec_kappa(n)) * Tc);
            S2 += Dn;
            Dm = Dc; Dc = Dn;
        }
        if (SP) {
            const float Pn = fmaf(qxp, Tc, fmaf(qx, Pc, -(float)rec_beta(n) * fmaf(q2p, Tm, q2 * Pm)));
            S3 = fmaf((float)rec_kappa(n + 1), Pn, S3);
            Pm = Pc; Pc = Pn;
        }
        Tm = Tc; Tc = Tn;
    }
    kahan_add(as, ac, h.w * rinv * S0);
    if (SP) kahan_add(ps, pc, h.w * rinv * S3);
    if (DLP) {
        const float Dp1 = fmaf(q2, Dm, (float)((2.0 * P + 1.0) * rec_kappa(P)) * Tc);
        const float S1 = 0.5f * (fmaf(-q2, S2, S2) + Dp1 + fmaf(q2, Dc, S0));
        const float a = fmaf(dx, nn.x, fmaf(dy, nn.y, dz * nn.z));
        const float b = fmaf(e.x, nn.x, fmaf(e.y, nn.y, e.z * nn.z));
        const float val = fmaf(-a, S1, fmaf(-a, qx, b) * S2);
        kahan_add(ds, dc, h.w * rinv * r2inv * val);
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
        double tx = 0, ty = 0, tz = 0, f2 = 0;
        if (SP) {
            const double4_32a tn = g.slot_n[it.slot_begin];
            tx = tn.x; ty = tn.y; tz = tn.z;
            f2 = 2.0 * fma(e.x, tx, fma(e.y, ty, e.z * tz));
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
                                  tx, ty, tz, f2, acc_s, acc_d, acc_p);
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
    double cx = 0, cy = 0, cz = 0, ex = 0, ey = 0, ez = 0, rho2 = 0, tx = 0, ty = 0, tz = 0, f2 = 0;
    if (active) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double4_32a e = g.slot_e[it.slot_begin + j];
        cx = c.x; cy = c.y; cz = c.z;
        ex = e.x; ey = e.y; ez = e.z; rho2 = e.w;
        if (SP) {
            const double4_32a tn = g.slot_n[it.slot_begin + j];
            tx = tn.x; ty = tn.y; tz = tn.z;
            f2 = 2.0 * fma(ex, tx, fma(ey, ty, ez * tz));
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
                                      tx, ty, tz, f2, acc_s, acc_d, acc_p);
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
            tn.w = 2.f * fmaf(e.x, tn.x, fmaf(e.y, tn.y, e.z * tn.z));
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
            tn.w = 2.f * fmaf(e.x, tn.x, fmaf(e.y, tn.y, e.z * tn.z));
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
