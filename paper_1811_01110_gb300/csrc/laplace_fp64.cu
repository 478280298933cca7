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

#include "laplace_items.cuh"

namespace tsqbx {
namespace {

template <int P, bool DLP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_fp64_kernel(const DevGeom g, const DevEval ev)
{
    __shared__ double tile[kWarpsPerBlock][DLP ? 7 : 4][kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;                       // whole warp leaves together
    laplace_fp64_item<P, DLP>(g, ev, g.items[item], tile[warp], lane);
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
