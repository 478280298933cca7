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
//   summing the Q' recurrence: sum_{n<=p} (2n+1) Q_n = (1-q2) sum_{n<=p} Q'_n
//   + Q'_{p+1} + q2 Q'_p.
//   S' (target-normal derivative of the single layer, n_t.grad_t G^(p)):
//        differentiate the recurrence along n_t -- qx' = (d.n_t)/R^2,
//        q2' = 2 (e.n_t)/R^2, T'_{n+1} = qx' T_n + qx T'_n - beta_n (q2' T_{n-1}
//        + q2 T'_{n-1}) -- and S' = (1/4pi) (1/R) sum_{n<=p} kappa_n T'_n.
// None of these forms divides by rho, so t = c needs no special case.
//
// Mapping: one warp per work item (a group's target chunk, L lanes per
// target); the group's sources are staged through shared memory in tiles of
// kTile; the L lanes of a target stride through each tile; per-target sums are
// combined by a segmented shuffle reduction in a fixed order (deterministic).
#include "laplace_launch.cuh"

namespace tsqbx {

int launch_laplace_fp64(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const bool dlp = (layers & 2u) != 0;
    if (layers & 4u) return launch_laplace_fp64_sp(p, dlp, g, e, s);
    return laplace_dispatch<false, false>(p, dlp, g, e, s);
}

}  // namespace tsqbx
