// conventional_helm.cu -- entry point of the Helmholtz conventional QBX path
// (kernels and arithmetic in conventional_helm.cuh): dispatch of the order to
// the translation unit that instantiates it.
#include "conventional_helm.cuh"

namespace tsqbx {

int launch_conventional_helm(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (g.n_conv_items == 0 && g.n_conv_eval == 0) return 0;
    if (p < 0 || p > kConvHelmMaxP) return (int)cudaErrorNotSupported;
    if (p <= 8) return launch_conv_helm_p0_8(p, layers, g, e, s);
    if (p <= 10) return launch_conv_helm_p9_10(p, layers, g, e, s);
    return launch_conv_helm_p11_12(p, layers, g, e, s);
}

}  // namespace tsqbx
