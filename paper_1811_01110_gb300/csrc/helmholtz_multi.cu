// helmholtz_multi.cu -- the Helmholtz single layer (arithmetic in
// helmholtz.cu) for 2..kMaxRhs densities in one launch.  Every per-pair
// quantity -- geometry, the Legendre and Hankel-factor recurrences, e^{ikR},
// the Clenshaw sum -- depends on the geometry, the order and the wavenumber
// alone, so the densities share it and each adds only its own complex weight
// (four FP64 operations per pair): n densities cost little more than one.
// This is what lets a serving loop run queued requests that share a plan, an
// order and a wavenumber as one evaluation.
#include "helmholtz_items.cuh"

namespace tsqbx {

int launch_helmholtz_multi(int p, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const auto ps = std::make_integer_sequence<int, 21>{};
    switch (e.n_rhs) {
    case 2: return dispatch_helm_multi<2>(p, g, e, s, ps);
    case 3: return dispatch_helm_multi<3>(p, g, e, s, ps);
    case 4: return dispatch_helm_multi<4>(p, g, e, s, ps);
    default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace tsqbx
