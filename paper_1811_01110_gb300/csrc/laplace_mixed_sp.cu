// laplace_mixed_sp.cu -- the mixed-precision Laplace kernels that also form S' = n_t.grad_t
// G^(p), the target-normal derivative of the single layer (kernel bodies in
// laplace_items.cuh; the arithmetic is described in laplace_mixed.cu).
#include "laplace_launch.cuh"

namespace tsqbx {

int launch_laplace_mixed_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return laplace_dispatch<true, true>(p, dlp, g, e, s);
}

}  // namespace tsqbx
