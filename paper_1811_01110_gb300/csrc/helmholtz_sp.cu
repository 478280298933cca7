// helmholtz_sp.cu -- the Helmholtz TSQBX kernels that also form S' =
// n_t.grad_t G_k^(p) (kernel in helmholtz_items.cuh; arithmetic in helmholtz.cu).
#include "helmholtz_items.cuh"

namespace tsqbx {

int launch_helmholtz_fp64_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return dispatch_helm<true>(p, dlp, g, e, s, std::make_integer_sequence<int, 21>{});
}

}  // namespace tsqbx
