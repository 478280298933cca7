// conventional_helm_p11_12.cu -- the Helmholtz conventional-path kernels
// (conventional_helm.cuh) for orders 11..12.
#include "conventional_helm.cuh"

namespace tsqbx {

int launch_conv_helm_p11_12(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_helm_range<11, 12>(p, layers, g, e, s);
}

}  // namespace tsqbx
