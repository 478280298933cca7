// conventional_p20.cu -- the conventional-path kernels (conventional.cuh)
// for orders 20..20.
#include "conventional.cuh"

namespace tsqbx {

int launch_conv_p20(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_range<20, 20>(p, layers, g, e, s);
}

}  // namespace tsqbx
