// conventional_helm_p9_10.cu -- the Helmholtz conventional-path kernels
// (conventional_helm.cuh) for orders 9..10.
#include "conventional_helm.cuh"

namespace tsqbx {

int launch_conv_helm_p9_10(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    return launch_conv_helm_range<9, 10>(p, layers, g, e, s);
}

}  // namespace tsqbx
