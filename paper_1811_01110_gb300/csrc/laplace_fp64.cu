// laplace_fp64.cu -- Laplace TSQBX kernels, every step in FP64.
//
// Per pair (target t with center c, source s; d = s - c, e = t - c):
//   R^2 = d.d, 1/R by rsqrt, qx = (d.e)/R^2 = (rho/R) cos g, q2 = rho^2/R^2
//   Q_n = (rho/R)^n P_n(cos g) through the scaled Bonnet recurrence
//   single layer  (Appendix A):  G^(p)          = (1/4pi) (1/R) sum_{n<=p} Q_n
//   double layer  (Appendix A):  n_s.grad_s G^(p) = (1/4pi) (1/R^3)
//        sum_{n<=p} [ -(n+1) a Q_n + (b - a qx) Q'_n ],   a = d.n_s, b = e.n_s,
//        Q'_n = (rho/R)^{n-1} P'_n,  Q'_{n+1} = q2 Q'_{n-1} + (2n+1) Q_n,
//   where sum (n+1) Q_n is recovered from sum Q'_n and Q'_p, Q'_{p+1} by
//   summing the Q' recurrence: sum_{n<=p} (2n+1) Q_n = (1-q2) S' + Q'_{p+1} + q2 Q'_p.
// Neither form divides by rho, so t = c needs no special case.
//
// Mapping: one warp per work item (a group's target chunk, L lanes per
// target); the group's sources are staged through shared memory in tiles of
// kTile; the L lanes of a target stride through each tile; per-target sums are
// combined by a segmented shuffle reduction in a fixed order (deterministic).
#include <utility>

#include "internal.cuh"

namespace tsqbx {
namespace {

template <int P, bool DLP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_fp64_kernel(const DevGeom g, const DevEval ev)
{
    constexpr int NF = DLP ? 7 : 4;
    __shared__ double tile[kWarpsPerBlock][NF][kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;                       // whole warp leaves together
    const Item it = g.items[item];
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
    const int64_t s0 = g.grp_off[it.group];
    const int src_hi = it.src_hi;
    double (*T)[kTile] = tile[warp];
    double acc_s = 0.0, acc_d = 0.0;

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
            for (int k = sub; k < cnt; k += L) {
                const double dx = T[0][k] - cx, dy = T[1][k] - cy, dz = T[2][k] - cz;
                const double wm = T[3][k];
                const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const double rinv = rsqrt(R2);
                const double r2inv = rinv * rinv;
                const double qx = fma(dx, ex, fma(dy, ey, dz * ez)) * r2inv;
                const double q2 = rho2 * r2inv;
                // n = 0 (and n = 1 when P >= 1)
                double S0 = 1.0, S2 = 0.0;
                double Tm = 1.0, Tc = 1.0, Dm = 0.0, Dc = 0.0;   // T_{n-1}, T_n, Q'_{n-1}, Q'_n
                if (P >= 1) { S0 += qx; S2 = 1.0; Tc = qx; Dc = 1.0; }
#pragma unroll
                for (int n = 1; n < P; ++n) {
                    const double Tn = fma(qx, Tc, -(rec_beta(n) * q2) * Tm);
                    S0 = fma(rec_kappa(n + 1), Tn, S0);
                    if (DLP) {
                        const double Dn = fma(q2, Dm, ((2.0 * n + 1.0) * rec_kappa(n)) * Tc);
                        S2 += Dn;
                        Dm = Dc; Dc = Dn;
                    }
                    Tm = Tc; Tc = Tn;
                }
                acc_s = fma(wm * rinv, S0, acc_s);
                if (DLP) {
                    const double Dp1 = fma(q2, Dm, ((2.0 * P + 1.0) * rec_kappa(P)) * Tc);
                    const double S1 = 0.5 * (fma(-q2, S2, S2) + Dp1 + fma(q2, Dc, S0));
                    const double a = fma(dx, T[4][k], fma(dy, T[5][k], dz * T[6][k]));
                    const double b = fma(ex, T[4][k], fma(ey, T[5][k], ez * T[6][k]));
                    const double val = fma(-a, S1, fma(-a, qx, b) * S2);
                    acc_d = fma(wm * rinv * r2inv, val, acc_d);
                }
            }
        }
        __syncwarp();
    }
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
    if (dlp) laplace_fp64_kernel<P, true><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(g, e);
    else     laplace_fp64_kernel<P, false><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(g, e);
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

int launch_laplace_fp64(int p, bool slp, bool dlp, const DevGeom &g, const DevEval &e,
                        cudaStream_t s)
{
    (void)slp;
    return dispatch(p, dlp, g, e, s, std::make_integer_sequence<int, 21>{});
}

}  // namespace tsqbx
