// laplace_multi.cu -- the Laplace single layer, or single and double layer,
// in FP64 (arithmetic in laplace_fp64.cu) for 2..kMaxRhs densities in one
// launch.  The per-pair kernel values of Appendix A's expansion -- geometry,
// 1/R, the sums over the orders -- depend on the geometry and the order
// alone, so the densities share them and each adds only its own w mu (two
// FP64 operations per pair and layer): n densities cost little more than
// one.  Same items, lanes and arithmetic as the single-density kernel of the
// plan's order form (one kernel per order, or the runtime-order kernel when
// DevGeom::p_unroll > 0), so each result is bit-identical to the evaluation
// of its density alone.
#include <utility>

#include "laplace_items.cuh"

namespace tsqbx {
namespace {

template <int P, bool DLP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_fp64_multi_kernel(const DevGeom g, const DevEval ev)
{
    extern __shared__ __align__(16) double smem_multi[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    double *T = smem_multi + (size_t)warp * multi_tile_rows(DLP) * g.tile;
    laplace_fp64_multi_item<P, DLP>(g, ev, g.items[item], g.item_walk[item], T, g.tile, lane);
}

template <int P>
int launch_multi_p(bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    static_assert((size_t)kWarpsPerBlock * multi_tile_rows(true) * kTileMax * sizeof(double) <= kSmemNoOptIn,
                  "staging tiles fit the default shared memory");
    const size_t smem = (size_t)kWarpsPerBlock * multi_tile_rows(dlp) * g.tile * sizeof(double);
    if (dlp) laplace_fp64_multi_kernel<P, true><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, s>>>(g, e);
    else     laplace_fp64_multi_kernel<P, false><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, s>>>(g, e);
    return (int)cudaGetLastError();
}

template <int... Ps>
int dispatch_multi(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s,
                   std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_multi_p<Ps>(dlp, g, e, s), 0) : 0), ...);
    return rc;
}

}  // namespace

int launch_laplace_fp64_multi(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (e.n_rhs < 2 || e.n_rhs > kMaxRhs || p < 0 || p > kPMax || e.p != p || !tile_depth_ok(g.tile))
        return (int)cudaErrorInvalidValue;
    switch (g.p_unroll) {
    case 0: return dispatch_multi(p, dlp, g, e, s, std::make_integer_sequence<int, kPMax + 1>{});
    case 1: return launch_multi_p<-1>(dlp, g, e, s);
    case 2: return launch_multi_p<-2>(dlp, g, e, s);
    case 4: return launch_multi_p<-4>(dlp, g, e, s);
    default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace tsqbx
