// laplace_df_items.cuh -- the double-float Laplace kernel (arithmetic in
// laplace_df64.cu) and its dispatch over p; laplace_df64.cu instantiates the
// single/double-layer variants, laplace_df64_sp.cu the ones that also form S'.
#pragma once

#include <utility>

#include "dfloat.cuh"
#include "internal.cuh"
#include "laplace_items.cuh"

namespace tsqbx {
namespace {

struct df3 {
    df x, y, z;
};

__device__ __forceinline__ df3 df3_from(double x, double y, double z)
{
    return {df_from_double(x), df_from_double(y), df_from_double(z)};
}

__device__ __forceinline__ df df_dot(const df3 &a, const df3 &b)
{
    return df_add(df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_mul(a.z, b.z));
}

// The pair's geometry in double-float: 1/R, 1/R^2, qx and q2.
__device__ __forceinline__ void pair_geom_df(const df3 &d, const df3 &e, df rho2, df &rinv, df &r2inv, df &qx,
                                             df &q2)
{
    const df R2 = df_dot(d, d);
    rinv = df_rsqrt(R2);
    r2inv = df_mul(rinv, rinv);
    qx = df_mul(df_dot(d, e), r2inv);
    q2 = df_mul(rho2, r2inv);
}

// The single layer's sum S = b_0 by Clenshaw's recurrence, as in pair_fp64.
template <int P>
__device__ __forceinline__ df slp_clenshaw_df(df qx, df q2)
{
    df b2 = df_of(df_const(rec_kappa(P)));
    df b1 = P >= 1 ? df_add(df_of(df_const(rec_kappa(P - 1))), df_mul(qx, b2)) : df{1.f, 0.f};
#pragma unroll
    for (int k = P - 2; k >= 0; --k) {
        const df bq = df_mul(df_of(df_const(rec_beta(k + 1))), q2);
        const df bk = df_sub(df_add(df_of(df_const(rec_kappa(k))), df_mul(qx, b1)), df_mul(bq, b2));
        b2 = b1; b1 = bk;
    }
    return b1;
}

// The Q'-recurrence sums in double-float, as qprime_sums_fp64: S2m, S2 =
// S2m + Q'_p, Q'_{p+1} and the single layer's S.
template <int P>
__device__ __forceinline__ void qprime_sums_df(df qx, df q2, df &S2m, df &S2, df &Qp1, df &S)
{
    const df one{1.f, 0.f};
    // the exact n = 1 step taken outside the loop, as in pair_fp64
    df Um{0.f, 0.f}, Uc = one;
    S2m = df{0.f, 0.f};
    if constexpr (P >= 2) { Um = one; Uc = qx; S2m = df_of(df_const(rec_lambda(1))); }
#pragma unroll
    for (int m = 2; m < P; ++m) {
        S2m = df_add(S2m, df_mul_c(df_const(rec_lambda(m)), Uc));
        const df gq = df_mul_c(df_const(rec_gamma(m)), q2);
        const df Un = df_sub(df_mul(qx, Uc), df_mul(gq, Um));
        Um = Uc; Uc = Un;
    }
    df Qp{0.f, 0.f};
    Qp1 = one;
    if (P >= 1) {
        Qp = df_mul_c(df_const(rec_lambda(P)), Uc);
        const df gq = df_mul_c(df_const(rec_gamma(P)), q2);
        Qp1 = df_mul_c(df_const(rec_lambda(P + 1)), df_sub(df_mul(qx, Uc), df_mul(gq, Um)));
    }
    S2 = df_add(S2m, Qp);
    // S = (1 - 2 qx + q2) S2 + Q'_{p+1} - q2 Q'_p
    const df c1 = df_add(df_sub(one, df_mul_f(qx, 2.f)), q2);
    S = df_add(df_mul(c1, S2), df_sub(Qp1, df_mul(q2, Qp)));
}

// One pair; tn = n_t and en = e.n_t (S' only).  Same two recurrences and
// closing sums as pair_fp64 (laplace_items.cuh), in double-float.
template <int P, bool DLP, bool SP>
__device__ __forceinline__ void pair_df(const df3 &d, const df3 &e, df rho2, df wm, const df3 &n, const df3 &tn,
                                        df en, df &acc_s, df &acc_d, df &acc_p)
{
    df rinv, r2inv, qx, q2;
    pair_geom_df(d, e, rho2, rinv, r2inv, qx, q2);
    const df wr = df_mul(wm, rinv);
    if constexpr (!DLP && !SP) {
        acc_s = df_add(acc_s, df_mul(wr, slp_clenshaw_df<P>(qx, q2)));
    } else {
        df S2m, S2, Qp1, S;
        qprime_sums_df<P>(qx, q2, S2m, S2, Qp1, S);
        acc_s = df_add(acc_s, df_mul(wr, S));
        const df wr3 = df_mul(wr, r2inv);
        if (DLP) {                     // (b - a) S2 - a Q'_{p+1}, as in pair_fp64
            const df a = df_dot(d, n);
            const df b = df_dot(e, n);
            const df val = df_sub(df_mul(df_sub(b, a), S2), df_mul(a, Qp1));
            acc_d = df_add(acc_d, df_mul(wr3, val));
        }
        if (SP) {
            const df dn = df_dot(d, tn);
            acc_p = df_add(acc_p, df_mul(wr3, df_sub(df_mul(dn, S2), df_mul(en, S2m))));
        }
    }
}

template <bool DLP, bool SP>
__device__ __forceinline__ void write_df_result(const DevGeom &g, const DevEval &ev, const Item &it, int j,
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

// Per-target target normal and e.n_t, both as double-floats.
__device__ __forceinline__ void df_target_normal(const DevGeom &g, int slot, const double4_32a &e4, df3 &tn, df &en)
{
    const double4_32a n = g.slot_n[slot];
    tn = df3_from(n.x, n.y, n.z);
    en = df_from_double(fma(e4.x, n.x, fma(e4.y, n.y, e4.z * n.z)));
}

// T: the warp's staging tile, rows of `tile` records: {x, y, z, w mu} hi and
// lo parts relative to the item's reference point and, for the double layer,
// the normal's hi and lo parts.
template <int P, bool DLP, bool SP>
__device__ __forceinline__ void laplace_df_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                const WalkStart &ws, float4 *T, const int tile, const int lane)
{
    ListWalk walk(g, ws);
    const int src_hi = it.src_hi;
    df acc_s{0.f, 0.f}, acc_d{0.f, 0.f}, acc_p{0.f, 0.f};
    const df3 zero3{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (it.n_tgt == 1) {                                   // direct loads, all 32 lanes
        const double4_32a c = g.slot_c[it.slot_begin];
        const double4_32a e4 = g.slot_e[it.slot_begin];
        const df3 e = df3_from(e4.x, e4.y, e4.z);
        const df rho2 = df_from_double(e4.w);
        df3 tn = zero3;
        df ent{0.f, 0.f};
        if (SP) df_target_normal(g, it.slot_begin, e4, tn, ent);
#pragma unroll 1
        for (int k = it.src_lo + lane; k < src_hi; k += 32) {
            int s = walk.at(k);
            double wmd = 0.0;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wmd = ev.wmu[s];
            const double4_32a pw = g.src_pw[s];
            const df3 d = df3_from(pw.x - c.x, pw.y - c.y, pw.z - c.z);
            df3 n = zero3;
            if (DLP) { const double4_32a nn = g.src_n[s]; n = df3_from(nn.x, nn.y, nn.z); }
            pair_df<P, DLP, SP>(d, e, rho2, df_from_double(wmd), n, tn, ent, acc_s, acc_d, acc_p);
        }
        double vs = df_to_double(acc_s), vd = df_to_double(acc_d), vp = df_to_double(acc_p);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            vs += __shfl_xor_sync(0xffffffffu, vs, off);
            if (DLP) vd += __shfl_xor_sync(0xffffffffu, vd, off);
            if (SP) vp += __shfl_xor_sync(0xffffffffu, vp, off);
        }
        if (lane == 0) write_df_result<DLP, SP>(g, ev, it, 0, vs, vd, vp);
        return;
    }
    const int L = it.L;
    const int j = lane / L, sub = lane - j * L;
    const bool active = j < it.n_tgt;
    const double4_32a ref = g.slot_c[it.slot_begin];      // item reference point
    df3 crel = zero3, e = zero3, tn = zero3;
    df rho2{0.f, 0.f}, ent{0.f, 0.f};
    if (active) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double4_32a e4 = g.slot_e[it.slot_begin + j];
        crel = df3_from(c.x - ref.x, c.y - ref.y, c.z - ref.z);
        e = df3_from(e4.x, e4.y, e4.z);
        rho2 = df_from_double(e4.w);
        if (SP) df_target_normal(g, it.slot_begin + j, e4, tn, ent);
    }
    float4 *const T0 = T, *const T1 = T + tile, *const T2 = T + 2 * tile, *const T3 = T + 3 * tile;
    for (int base = it.src_lo; base < src_hi; base += tile) {
        const int cnt = min(tile, src_hi - base);
        for (int k = lane; k < cnt; k += 32) {
            int s = walk.at(base + k);
            double wmd = 0.0;
            if ((unsigned)s >= (unsigned)g.n_src) { atomicOr(ev.status, 1); s = 0; }
            else wmd = ev.wmu[s];
            const double4_32a pw = g.src_pw[s];
            const df3 r = df3_from(pw.x - ref.x, pw.y - ref.y, pw.z - ref.z);
            const df w = df_from_double(wmd);
            T0[k] = make_float4(r.x.hi, r.y.hi, r.z.hi, w.hi);
            T1[k] = make_float4(r.x.lo, r.y.lo, r.z.lo, w.lo);
            if (DLP) {
                const double4_32a nn = g.src_n[s];
                const df3 n = df3_from(nn.x, nn.y, nn.z);
                T2[k] = make_float4(n.x.hi, n.y.hi, n.z.hi, 0.f);
                T3[k] = make_float4(n.x.lo, n.y.lo, n.z.lo, 0.f);
            }
        }
        __syncwarp();
        if (active) {
            for (int k = sub; k < cnt; k += L) {
                const float4 a = T0[k], b = T1[k];
                const df3 d{df_sub(df{a.x, b.x}, crel.x), df_sub(df{a.y, b.y}, crel.y),
                            df_sub(df{a.z, b.z}, crel.z)};
                df3 n = zero3;
                if (DLP) {
                    const float4 c = T2[k], h = T3[k];
                    n = df3{{c.x, h.x}, {c.y, h.y}, {c.z, h.z}};
                }
                pair_df<P, DLP, SP>(d, e, rho2, df{a.w, b.w}, n, tn, ent, acc_s, acc_d, acc_p);
            }
        }
        __syncwarp();
    }
    double vs = df_to_double(acc_s), vd = df_to_double(acc_d), vp = df_to_double(acc_p);
    for (int off = 1; off < L; off <<= 1) {
        const double ts = __shfl_down_sync(0xffffffffu, vs, off);
        const double td = DLP ? __shfl_down_sync(0xffffffffu, vd, off) : 0.0;
        const double tp = SP ? __shfl_down_sync(0xffffffffu, vp, off) : 0.0;
        if (sub + off < L) { vs += ts; vd += td; vp += tp; }
    }
    if (active && sub == 0) write_df_result<DLP, SP>(g, ev, it, j, vs, vd, vp);
}

// BOTH_PIPES: items with (index mod 20) < g.fp64_share run the native FP64
// item body (laplace_items.cuh) on the FP64 pipe, the others the
// double-float body on the FP32 pipes.  The split is by item index, so the
// two kinds are spread over the whole launch and share every SM, and each
// target's result comes from the same body on every run.  The FP64 body
// reads the same arrays (FP64 sources, w mu, target records) and its
// staging tile fits in the double-float one (DLP: 7 doubles vs 4 float4 per
// source; otherwise 4 doubles vs 2 float4).
template <int P, bool DLP, bool SP, bool BOTH_PIPES = false>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_df_kernel(const DevGeom g, const DevEval ev)
{
    extern __shared__ __align__(16) float4 smem_df[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    float4 *T = smem_df + (size_t)warp * (DLP ? 4 : 2) * g.tile;
    static_assert((DLP ? 7 : 4) * sizeof(double) <= (DLP ? 4 : 2) * sizeof(float4), "FP64 tile fits");
    if constexpr (BOTH_PIPES) {
        if ((int)(item % 20) < g.fp64_share) {
            laplace_fp64_item<P, DLP, SP>(g, ev, g.items[item], g.item_walk[item], reinterpret_cast<double *>(T),
                                          g.tile, lane);
            return;
        }
    }
    laplace_df_item<P, DLP, SP>(g, ev, g.items[item], g.item_walk[item], T, g.tile, lane);
}

template <bool SP, int P>
int launch_df_p(bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    if (!tile_depth_ok(g.tile) || g.fp64_share < 0 || g.fp64_share > 20) return (int)cudaErrorInvalidValue;
    static_assert((size_t)kWarpsPerBlock * 4 * kTileMax * sizeof(float4) <= kSmemNoOptIn,
                  "staging tiles fit the default shared memory");
    const size_t smem = (size_t)kWarpsPerBlock * (dlp ? 4 : 2) * g.tile * sizeof(float4);
    const unsigned b = (unsigned)blocks, t = kWarpsPerBlock * 32;
    if (g.fp64_share > 0) {
        if (dlp) laplace_df_kernel<P, true, SP, true><<<b, t, smem, s>>>(g, e);
        else     laplace_df_kernel<P, false, SP, true><<<b, t, smem, s>>>(g, e);
    } else {
        if (dlp) laplace_df_kernel<P, true, SP><<<b, t, smem, s>>>(g, e);
        else     laplace_df_kernel<P, false, SP><<<b, t, smem, s>>>(g, e);
    }
    return (int)cudaGetLastError();
}

template <bool SP, int... Ps>
int dispatch_df(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s,
                std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_df_p<SP, Ps>(dlp, g, e, s), 0) : 0), ...);
    return rc;
}

}  // namespace

// Defined in laplace_df64_sp.cu.
int launch_laplace_df64_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s);

}  // namespace tsqbx
