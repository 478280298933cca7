// laplace_df64_sp.cu -- the double-float Laplace kernels that also form
// S' = n_t.grad_t G^(p) (kernel body in laplace_df_items.cuh; arithmetic in
// laplace_df64.cu).
#include "laplace_df_items.cuh"

namespace tsqbx {

int launch_laplace_df64_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return dispatch_df<true>(p, dlp, g, e, s, std::make_integer_sequence<int, 21>{});
}

}  // namespace tsqbx
