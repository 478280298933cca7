// conventional_helm_p0_8.cu -- the Helmholtz conventional-path kernels
// (conventional_helm.cuh) for orders 0..8.
#include "conventional_helm.cuh"

namespace tsqbx {

int launch_conv_helm_p0_8(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_helm_range<0, 8>(p, layers, g, e, s);
}

}  // namespace tsqbx
