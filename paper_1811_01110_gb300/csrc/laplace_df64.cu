// laplace_df64.cu -- Laplace TSQBX kernels with FP64-class accuracy computed
// in double-float arithmetic (dfloat.cuh) on the FP32 pipes.
//
// Same expansion, recurrences and warp mapping as laplace_fp64.cu (Appendix
// A; the scaled Bonnet recurrence for the single layer alone, the Q'-only
// recurrence with its closing sums when the double layer or S' is formed),
// every quantity a double-float.  Geometry: each item picks a reference point (its first
// target's center) and forms s - ref and c - ref in FP64 before splitting
// them into double-floats, so d = s - c keeps ~48 significant bits relative
// to |d| itself.  The recurrence constants are exact double-float splits of
// their double values (products by the ones that are floats take the cheaper
// double-word-times-float algorithm).  Per-lane sums are double-floats; lanes
// of a target are combined in FP64.
//
// Both pipes (DevGeom::fp64_share, tuned): items with index mod 20 below the
// share run the native FP64 item body in the same launch, on the FP64 pipe
// that the double-float items leave mostly idle.
#include "laplace_df_items.cuh"

namespace tsqbx {

int launch_laplace_df64(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const bool dlp = (layers & 2u) != 0;
    if (layers & 4u) return launch_laplace_df64_sp(p, dlp, g, e, s);
    return dispatch_df<false>(p, dlp, g, e, s, std::make_integer_sequence<int, 21>{});
}

}  // namespace tsqbx
