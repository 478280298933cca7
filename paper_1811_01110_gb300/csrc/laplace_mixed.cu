// laplace_mixed.cu -- Laplace TSQBX kernels in mixed precision.
//
// Same expansion, recurrences and warp mapping as laplace_fp64.cu (Appendix
// A; the scaled Bonnet recurrence for the single layer alone, the Q'-only
// recurrence with its closing sums otherwise), with the arithmetic split as:
//  * coordinates arrive as float-float pairs (hi + lo, formed from the FP64
//    inputs when the plan is built); s - c is formed as (s_hi - c_hi) +
//    (s_lo - c_lo), accurate to FP32 rounding of the difference itself, so
//    nearby sources lose no digits to cancellation;
//  * e = t - c and rho^2 are formed in FP64 at plan time and rounded once;
//  * the geometry ratios, 1/R and 1/R^2 (each one special-function
//    instruction; 1/R^2 its own reciprocal, not (1/R)^2, when the double
//    layer or S' is formed: the Q' recurrence amplifies the error of qx and
//    q2 with the order) and the recurrence run in FP32;
//  * each lane sums a shared-memory tile's pairs in plain FP32 and adds the
//    tile sum to Kahan-compensated FP32 sums (single-target items compensate
//    every pair); the L lanes of a target are combined in double-float on the
//    FP32 pipes, and the output is FP64;
//  * each lane takes two sources at a time and runs every FP32 operation as
//    a packed f32x2 instruction (f32x2.cuh): the same flops in half the issue
//    slots.  The staged tile holds sources pairwise, so one 16-byte shared
//    load gives two packed operands.
#include "laplace_launch.cuh"

namespace tsqbx {

int launch_laplace_mixed(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const bool dlp = (layers & 2u) != 0;
    if (layers & 4u) return launch_laplace_mixed_sp(p, dlp, g, e, s);
    return laplace_dispatch<true, false>(p, dlp, g, e, s);
}

}  // namespace tsqbx
