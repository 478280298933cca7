// conventional_p18_19.cu -- the conventional-path kernels (conventional.cuh)
// for orders 18..19.
#include "conventional.cuh"

namespace tsqbx {

int launch_conv_p18_19(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_range<18, 19>(p, layers, g, e, s);
}

}  // namespace tsqbx
