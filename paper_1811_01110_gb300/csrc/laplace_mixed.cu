// laplace_mixed.cu -- Laplace TSQBX kernels in mixed precision.
//
// Same expansion and warp mapping as laplace_fp64.cu (Appendix A; scaled
// Bonnet recurrence Q_n = (rho/R)^n P_n), with the arithmetic split as:
//  * coordinates arrive as float-float pairs (hi + lo, formed from the FP64
//    inputs when the plan is built); s - c is formed as (s_hi - c_hi) +
//    (s_lo - c_lo), accurate to FP32 rounding of the difference itself, so
//    nearby sources lose no digits to cancellation;
//  * e = t - c and rho^2 are formed in FP64 at plan time and rounded once;
//  * the geometry ratios, 1/R (rsqrtf) and the recurrence run in FP32;
//  * each lane keeps Kahan-compensated FP32 sums; the L lanes of a target are
//    combined in FP64, and the output is FP64.
#include <utility>

#include "internal.cuh"

namespace tsqbx {
namespace {

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

template <int P, bool DLP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_mixed_kernel(const DevGeom g, const DevEval ev)
{
    constexpr int NF = DLP ? 3 : 2;
    __shared__ float4 tile[kWarpsPerBlock][NF][kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    const Item it = g.items[item];
    const int L = it.L;
    const int j = lane / L, sub = lane - j * L;
    const bool active = j < it.n_tgt;
    float4 ch = make_float4(0, 0, 0, 0), cl = ch, e = ch;
    if (active) {
        ch = g.slot_chi[it.slot_begin + j];
        cl = g.slot_clo[it.slot_begin + j];
        e = g.slot_ef[it.slot_begin + j];
    }
    const int64_t s0 = g.grp_off[it.group];
    const int src_hi = it.src_hi;
    float4 (*T)[kTile] = tile[warp];
    float as = 0.f, ac = 0.f, ds = 0.f, dc = 0.f;     // Kahan pairs (single, double layer)

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
            for (int k = sub; k < cnt; k += L) {
                const float4 h = T[0][k], l = T[1][k];
                const float dx = __fadd_rn(__fsub_rn(h.x, ch.x), __fsub_rn(l.x, cl.x));
                const float dy = __fadd_rn(__fsub_rn(h.y, ch.y), __fsub_rn(l.y, cl.y));
                const float dz = __fadd_rn(__fsub_rn(h.z, ch.z), __fsub_rn(l.z, cl.z));
                const float R2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float rinv = rsqrtf(R2);
                const float r2inv = rinv * rinv;
                const float qx = fmaf(dx, e.x, fmaf(dy, e.y, dz * e.z)) * r2inv;
                const float q2 = e.w * r2inv;
                float S0 = 1.f, S2 = 0.f;
                float Tm = 1.f, Tc = 1.f, Dm = 0.f, Dc = 0.f;
                if (P >= 1) { S0 += qx; S2 = 1.f; Tc = qx; Dc = 1.f; }
#pragma unroll
                for (int n = 1; n < P; ++n) {
                    const float Tn = fmaf(qx, Tc, -((float)rec_beta(n) * q2) * Tm);
                    S0 = fmaf((float)rec_kappa(n + 1), Tn, S0);
                    if (DLP) {
                        const float Dn = fmaf(q2, Dm, (float)((2.0 * n + 1.0) * rec_kappa(n)) * Tc);
                        S2 += Dn;
                        Dm = Dc; Dc = Dn;
                    }
                    Tm = Tc; Tc = Tn;
                }
                kahan_add(as, ac, h.w * rinv * S0);
                if (DLP) {
                    const float4 nn = T[2][k];
                    const float Dp1 = fmaf(q2, Dm, (float)((2.0 * P + 1.0) * rec_kappa(P)) * Tc);
                    const float S1 = 0.5f * (fmaf(-q2, S2, S2) + Dp1 + fmaf(q2, Dc, S0));
                    const float a = fmaf(dx, nn.x, fmaf(dy, nn.y, dz * nn.z));
                    const float b = fmaf(e.x, nn.x, fmaf(e.y, nn.y, e.z * nn.z));
                    const float val = fmaf(-a, S1, fmaf(-a, qx, b) * S2);
                    kahan_add(ds, dc, h.w * rinv * r2inv * val);
                }
            }
        }
        __syncwarp();
    }
    double acc_s = (double)as - (double)ac;
    double acc_d = (double)ds - (double)dc;
    for (int off = 1; off < L; off <<= 1) {
        const double vs = __shfl_down_sync(0xffffffffu, acc_s, off);
        const double vd = __shfl_down_sync(0xffffffffu, acc_d, off);
        if (sub + off < L) { acc_s += vs; acc_d += vd; }
    }
    if (active && sub == 0) {
        if (it.part < 0) {
            const int t = g.slot_tgt[it.slot_begin + j];
            if (ev.out_slp) ev.out_slp[t] = acc_s * kInv4Pi;
            if (DLP && ev.out_dlp) ev.out_dlp[t] = acc_d * kInv4Pi;
        } else {
            ev.part_slp[it.part + j] = acc_s * kInv4Pi;
            if (DLP) ev.part_dlp[it.part + j] = acc_d * kInv4Pi;
        }
    }
}

template <int P>
int launch_p(bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    if (dlp) laplace_mixed_kernel<P, true><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(g, e);
    else     laplace_mixed_kernel<P, false><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(g, e);
    return (int)cudaGetLastError();
}

template <int... Ps>
int dispatch(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s,
             std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_p<Ps>(dlp, g, e, s), 0) : 0), ...);
    return rc;
}

}  // namespace

int launch_laplace_mixed(int p, bool slp, bool dlp, const DevGeom &g, const DevEval &e,
                         cudaStream_t s)
{
    (void)slp;
    return dispatch(p, dlp, g, e, s, std::make_integer_sequence<int, 21>{});
}

}  // namespace tsqbx
