// constants_shim.cu -- test-only C entry points to the recurrence constants
// and conventional-QBX weights that the kernels take from their headers
// (internal.cuh, conventional.cuh, conventional_helm.cuh: host/device
// constexpr functions, compiled here unchanged), so that the CPU tests can
// check them against closed forms and addition theorems.
#include "../../paper_1811_01110_gb300/csrc/conventional_helm.cuh"
#include "../../paper_1811_01110_gb300/csrc/dfloat.cuh"

#define SHIM_API extern "C" __attribute__((visibility("default")))

SHIM_API double shim_rec_kappa(int n) { return tsqbx::rec_kappa(n); }
SHIM_API double shim_rec_beta(int n) { return tsqbx::rec_beta(n); }
SHIM_API double shim_rec_lambda(int n) { return tsqbx::rec_lambda(n); }
SHIM_API double shim_rec_gamma(int n) { return tsqbx::rec_gamma(n); }
SHIM_API double shim_conv_eps(int n, int m) { return tsqbx::conv_eps(n, m); }
SHIM_API double shim_conv_weight(int n, int m) { return tsqbx::conv_weight_table().w[n][m]; }
SHIM_API double shim_conv_helm_weight(int n, int m) { return tsqbx::conv_helm_weight_table().w[n][m]; }
SHIM_API int shim_conv_helm_max_p(void) { return tsqbx::kConvHelmMaxP; }
SHIM_API double shim_inv_4pi(void) { return tsqbx::kInv4Pi; }
SHIM_API void shim_df_const(double v, float *hi, float *lo)
{
    const tsqbx::dfc c = tsqbx::df_const(v);
    *hi = c.hi;
    *lo = c.lo;
}
