// conventional_p11_13.cu -- the conventional-path kernels (conventional.cuh)
// for orders 11..13.
#include "conventional.cuh"

namespace tsqbx {

int launch_conv_p11_13(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_range<11, 13>(p, layers, g, e, s);
}

}  // namespace tsqbx
