// laplace_fp64_sp.cu -- the FP64 Laplace kernels that also form S' = n_t.grad_t
// G^(p), the target-normal derivative of the single layer (kernel bodies in
// laplace_items.cuh; the arithmetic is described in laplace_fp64.cu).
#include "laplace_launch.cuh"

namespace tsqbx {

int launch_laplace_fp64_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return laplace_dispatch<false, true>(p, dlp, g, e, s);
}

}  // namespace tsqbx
