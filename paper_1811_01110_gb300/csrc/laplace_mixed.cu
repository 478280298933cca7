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

#include "laplace_items.cuh"

namespace tsqbx {
namespace {


template <int P, bool DLP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_mixed_kernel(const DevGeom g, const DevEval ev)
{
    __shared__ float4 tile[kWarpsPerBlock][DLP ? 3 : 2][kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    laplace_mixed_item<P, DLP>(g, ev, g.items[item], tile[warp], lane);
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
