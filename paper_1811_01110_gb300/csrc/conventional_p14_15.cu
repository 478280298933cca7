// conventional_p14_15.cu -- the conventional-path kernels (conventional.cuh)
// for orders 14..15.
#include "conventional.cuh"

namespace tsqbx {

int launch_conv_p14_15(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_range<14, 15>(p, layers, g, e, s);
}

}  // namespace tsqbx
