// conventional_p16_17.cu -- the conventional-path kernels (conventional.cuh)
// for orders 16..17.
#include "conventional.cuh"

namespace tsqbx {

int launch_conv_p16_17(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_range<16, 17>(p, layers, g, e, s);
}

}  // namespace tsqbx
