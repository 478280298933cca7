// conventional.cu -- entry point of the conventional QBX path (kernels and
// their arithmetic in conventional.cuh): dispatch of the order to the
// translation unit that instantiates it.
#include "conventional.cuh"

namespace tsqbx {

int launch_conventional(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (g.n_conv_items == 0 && g.n_conv_eval == 0) return 0;
    if (p < 0 || p > 20) return (int)cudaErrorInvalidValue;
    if (p <= 10) return launch_conv_p0_10(p, layers, g, e, s);
    if (p <= 13) return launch_conv_p11_13(p, layers, g, e, s);
    if (p <= 15) return launch_conv_p14_15(p, layers, g, e, s);
    if (p <= 17) return launch_conv_p16_17(p, layers, g, e, s);
    if (p <= 19) return launch_conv_p18_19(p, layers, g, e, s);
    return launch_conv_p20(p, layers, g, e, s);
}

}  // namespace tsqbx
