// laplace_fp64.cu -- Laplace TSQBX kernels, every step in FP64.
//
// Per pair (target t with center c, source s; d = s - c, e = t - c):
//   R^2 = d.d, 1/R by rsqrt, qx = (d.e)/R^2 = (rho/R) cos g, q2 = rho^2/R^2,
//   Q_n = (rho/R)^n P_n(cos g), Q'_n = (rho/R)^{n-1} P_n'(cos g);
//   single layer  (Appendix A):  G^(p)          = (1/4pi) (1/R) sum_{n<=p} Q_n
//   double layer  (Appendix A):  n_s.grad_s G^(p) = (1/4pi) (1/R^3)
//        sum_{n<=p} [ -(n+1) a Q_n + (b - a qx) Q'_n ],   a = d.n_s, b = e.n_s,
//   S'            (Appendix A):  n_t.grad_t G^(p) = (1/4pi) (1/R^3)
//        [ (d.n_t) sum_{n<=p} Q'_n - (e.n_t) sum_{n<p} Q'_n ].
// The single layer alone runs the scaled Bonnet recurrence for Q_n.  With
// the double layer or S', one recurrence for Q'_n alone (Gegenbauer C^(3/2))
// gives every sum: sum Q_n and sum (n+1) Q_n follow from sum Q'_n, Q'_p and
// Q'_{p+1} by two Legendre identities (pair_fp64 in laplace_items.cuh), so the
// three layers cost one recurrence of three operations per order (from n = 2:
// the n = 1 step is exact).  None of these forms divides by rho, so t = c
// needs no special case.
//
// Order forms: one kernel per order p with the recurrences fully unrolled
// (DevGeom::p_unroll = 0), or one kernel for every order whose loop over n
// is unrolled by p_unroll = 1, 2 or 4, its coefficients read from a
// constant-memory table (laplace_items.cuh); the autotuner picks.
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
