// laplace_df64_multi.cu -- the double-float Laplace single layer, or single
// and double layer (arithmetic in laplace_df64.cu), for 2..kMaxRhs densities
// in one launch.  As in laplace_multi.cu, the per-pair kernel values depend
// on the geometry and the order alone; each density adds its own w mu (per
// layer two double-float products and one double-float sum per pair).  Same
// items, lanes, arithmetic and both-pipes split (DevGeom::fp64_share) as the
// single-density double-float kernel, so each result is bit-identical to the
// evaluation of its density alone.
#include <utility>

#include "laplace_df_items.cuh"

namespace tsqbx {
namespace {

template <int P, bool DLP>
__device__ __forceinline__ void pair_df_multi(const df3 &d, const df3 &e, df rho2, const df3 &n,
                                              const df (&wm)[kMaxRhs], df (&acc)[kMaxRhs], df (&acc_d)[kMaxRhs],
                                              int nr)
{
    df rinv, r2inv, qx, q2;
    pair_geom_df(d, e, rho2, rinv, r2inv, qx, q2);
    if constexpr (!DLP) {
        const df S = slp_clenshaw_df<P>(qx, q2);
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r)
            if (r < nr) acc[r] = df_add(acc[r], df_mul(df_mul(wm[r], rinv), S));
    } else {
        df S2m, S2, Qp1, S;
        qprime_sums_df<P>(qx, q2, S2m, S2, Qp1, S);
        const df a = df_dot(d, n);
        const df b = df_dot(e, n);
        const df val = df_sub(df_mul(df_sub(b, a), S2), df_mul(a, Qp1));
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r)
            if (r < nr) {
                const df wr = df_mul(wm[r], rinv);
                acc[r] = df_add(acc[r], df_mul(wr, S));
                acc_d[r] = df_add(acc_d[r], df_mul(df_mul(wr, r2inv), val));
            }
    }
}

// laplace_df_item<P, DLP, false> with one double-float accumulator per
// density and layer.  T: rows of `tile` float4 records, {x, y, z, w mu_0} hi
// parts and lo parts (relative to the item's reference point), the hi, lo
// pairs of {w mu_1, w mu_2} and {w mu_3, unused}, then (DLP) the normal's hi
// and lo parts.
template <int P, bool DLP>
__device__ __forceinline__ void laplace_df_multi_item(const DevGeom &g, const DevEval &ev, const Item &it,
                                                      const WalkStart &ws, float4 *T, const int tile,
                                                      const int lane)
{
    ListWalk walk(g, ws);
    const int src_hi = it.src_hi;
    const int nr = ev.n_rhs;
    const int64_t stride = ev.rhs_src_stride;
    const df zero{0.f, 0.f};
    const df3 zero3{zero, zero, zero};
    df acc[kMaxRhs] = {zero, zero, zero, zero}, acc_d[kMaxRhs] = {zero, zero, zero, zero};
    if (it.n_tgt == 1) {                                   // direct loads, all 32 lanes
        const double4_32a c = g.slot_c[it.slot_begin];
        const double4_32a e4 = g.slot_e[it.slot_begin];
        const df3 e = df3_from(e4.x, e4.y, e4.z);
        const df rho2 = df_from_double(e4.w);
#pragma unroll 1
        for (int k = it.src_lo + lane; k < src_hi; k += 32) {
            int s = walk.at(k);
            const bool ok = (unsigned)s < (unsigned)g.n_src;
            if (!ok) { atomicOr(ev.status, 1); s = 0; }
            df wm[kMaxRhs];
#pragma unroll
            for (int r = 0; r < kMaxRhs; ++r) wm[r] = df_from_double(ok && r < nr ? ev.wmu[r * stride + s] : 0.0);
            const double4_32a pw = g.src_pw[s];
            const df3 d = df3_from(pw.x - c.x, pw.y - c.y, pw.z - c.z);
            df3 n = zero3;
            if (DLP) { const double4_32a nn = g.src_n[s]; n = df3_from(nn.x, nn.y, nn.z); }
            pair_df_multi<P, DLP>(d, e, rho2, n, wm, acc, acc_d, nr);
        }
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r)
            if (r < nr) {
                double v = df_to_double(acc[r]), vd = df_to_double(acc_d[r]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    v += __shfl_xor_sync(0xffffffffu, v, off);
                    if (DLP) vd += __shfl_xor_sync(0xffffffffu, vd, off);
                }
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
    const double4_32a ref = g.slot_c[it.slot_begin];      // item reference point
    df3 crel = zero3, e = zero3;
    df rho2 = zero;
    if (active) {
        const double4_32a c = g.slot_c[it.slot_begin + j];
        const double4_32a e4 = g.slot_e[it.slot_begin + j];
        crel = df3_from(c.x - ref.x, c.y - ref.y, c.z - ref.z);
        e = df3_from(e4.x, e4.y, e4.z);
        rho2 = df_from_double(e4.w);
    }
    float4 *const T0 = T, *const T1 = T + tile, *const T2 = T + 2 * tile, *const T3 = T + 3 * tile;
    float4 *const T4 = T + 4 * tile, *const T5 = T + 5 * tile;     // DLP only
    for (int base = it.src_lo; base < src_hi; base += tile) {
        const int cnt = min(tile, src_hi - base);
        for (int k = lane; k < cnt; k += 32) {
            int s = walk.at(base + k);
            const bool ok = (unsigned)s < (unsigned)g.n_src;
            if (!ok) { atomicOr(ev.status, 1); s = 0; }
            const double4_32a pw = g.src_pw[s];
            const df3 r = df3_from(pw.x - ref.x, pw.y - ref.y, pw.z - ref.z);
            const df w0 = df_from_double(ok ? ev.wmu[s] : 0.0);
            const df w1 = df_from_double(ok ? ev.wmu[stride + s] : 0.0);
            const df w2 = nr > 2 ? df_from_double(ok ? ev.wmu[2 * stride + s] : 0.0) : zero;
            T0[k] = make_float4(r.x.hi, r.y.hi, r.z.hi, w0.hi);
            T1[k] = make_float4(r.x.lo, r.y.lo, r.z.lo, w0.lo);
            T2[k] = make_float4(w1.hi, w1.lo, w2.hi, w2.lo);
            if (nr > 3) {
                const df w3 = df_from_double(ok ? ev.wmu[3 * stride + s] : 0.0);
                T3[k] = make_float4(w3.hi, w3.lo, 0.f, 0.f);
            }
            if (DLP) {
                const double4_32a nn = g.src_n[s];
                const df3 n = df3_from(nn.x, nn.y, nn.z);
                T4[k] = make_float4(n.x.hi, n.y.hi, n.z.hi, 0.f);
                T5[k] = make_float4(n.x.lo, n.y.lo, n.z.lo, 0.f);
            }
        }
        __syncwarp();
        if (active) {
            for (int k = sub; k < cnt; k += L) {
                const float4 a = T0[k], b = T1[k], w12 = T2[k];
                const float4 w3 = nr > 3 ? T3[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const df3 d{df_sub(df{a.x, b.x}, crel.x), df_sub(df{a.y, b.y}, crel.y),
                            df_sub(df{a.z, b.z}, crel.z)};
                df3 n = zero3;
                if (DLP) {
                    const float4 c = T4[k], h = T5[k];
                    n = df3{{c.x, h.x}, {c.y, h.y}, {c.z, h.z}};
                }
                const df wm[kMaxRhs] = {df{a.w, b.w}, df{w12.x, w12.y}, df{w12.z, w12.w}, df{w3.x, w3.y}};
                pair_df_multi<P, DLP>(d, e, rho2, n, wm, acc, acc_d, nr);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < kMaxRhs; ++r)
        if (r < nr) {
            double v = df_to_double(acc[r]), vd = df_to_double(acc_d[r]);
            for (int off = 1; off < L; off <<= 1) {
                const double t = __shfl_down_sync(0xffffffffu, v, off);
                const double td = DLP ? __shfl_down_sync(0xffffffffu, vd, off) : 0.0;
                if (sub + off < L) { v += t; vd += td; }
            }
            if (active && sub == 0) {
                write_multi_result<false>(g, ev, it, j, r, v);
                if (DLP) write_multi_result<true>(g, ev, it, j, r, vd);
            }
        }
}

// Staging rows (float4) of a double-float multi-density item.
__host__ __device__ constexpr int df_multi_rows(bool dlp) { return dlp ? 6 : 4; }

// Items with (index mod 20) < g.fp64_share run the native FP64 body, as in
// laplace_df_kernel; its staging rows (multi_tile_rows doubles per source)
// fit in the double-float ones.
template <int P, bool DLP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_df_multi_kernel(const DevGeom g, const DevEval ev)
{
    extern __shared__ __align__(16) float4 smem_dfm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    float4 *T = smem_dfm + (size_t)warp * df_multi_rows(DLP) * g.tile;
    static_assert(multi_tile_rows(DLP) * sizeof(double) <= df_multi_rows(DLP) * sizeof(float4),
                  "FP64 multi tile fits");
    if ((int)(item % 20) < g.fp64_share) {
        laplace_fp64_multi_item<P, DLP>(g, ev, g.items[item], g.item_walk[item], reinterpret_cast<double *>(T),
                                        g.tile, lane);
        return;
    }
    laplace_df_multi_item<P, DLP>(g, ev, g.items[item], g.item_walk[item], T, g.tile, lane);
}

template <int P>
int launch_df_multi_p(bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    static_assert((size_t)kWarpsPerBlock * df_multi_rows(true) * kTileMax * sizeof(float4) <= kSmemNoOptIn,
                  "staging tiles fit the default shared memory");
    const size_t smem = (size_t)kWarpsPerBlock * df_multi_rows(dlp) * g.tile * sizeof(float4);
    const unsigned b = (unsigned)blocks, t = kWarpsPerBlock * 32;
    if (dlp) laplace_df_multi_kernel<P, true><<<b, t, smem, s>>>(g, e);
    else     laplace_df_multi_kernel<P, false><<<b, t, smem, s>>>(g, e);
    return (int)cudaGetLastError();
}

template <int... Ps>
int dispatch_df_multi(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s,
                      std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_df_multi_p<Ps>(dlp, g, e, s), 0) : 0), ...);
    return rc;
}

}  // namespace

int launch_laplace_df64_multi(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (e.n_rhs < 2 || e.n_rhs > kMaxRhs || !tile_depth_ok(g.tile) || g.fp64_share < 0 || g.fp64_share > 20)
        return (int)cudaErrorInvalidValue;
    return dispatch_df_multi(p, dlp, g, e, s, std::make_integer_sequence<int, kPMax + 1>{});
}

}  // namespace tsqbx
