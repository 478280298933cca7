// conventional_p0_10.cu -- the conventional-path kernels (conventional.cuh)
// for orders 0..10.
#include "conventional.cuh"

namespace tsqbx {

int launch_conv_p0_10(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_range<0, 10>(p, layers, g, e, s);
}

}  // namespace tsqbx
