// helmholtz.cu -- Helmholtz TSQBX kernels (single layer, double layer, S'),
// FP64 throughout.
//
// Appendix A:  G_k^(p)(t,s) = ik/(4pi) sum_{n<=p} (2n+1) j_n(k rho) h_n(kR) P_n(cos g)
// with rho = |t-c|, R = |s-c|, h_n = h_n^(1).
//  * per target (once per work item): j_n(k rho), n <= p, by Miller's downward
//    recurrence f_{n-1} = (2n+1)/z f_n - f_{n+1} (DLMF 10.51.1), started
//    p + 20 + ceil(z) terms up and normalised against j_0 = sin z/z or
//    j_1 = sin z/z^2 - cos z/z, whichever is larger;
//  * per pair: h_n(z) = e^{iz} g_n(z), z = kR, where g_n obeys the same
//    recurrence (DLMF 10.51.1) with g_0 = -i/z, g_1 = -(1/z + i/z^2)
//    (DLMF 10.49.6 with 10.47.5), so one sincos per pair serves every order;
//  * P_n(cos g) by the scaled Bonnet recurrence with q = 1 (P_n = kappa_n T_n).
//  * double layer, n_s.grad_s: R changes by a/R (a = d.n_s) and cos g by
//    (1/R)((e.n_s)/rho - (a/R) cos g); h_n' = e^{iz}(g_{n-1} - (n+1)/z g_n)
//    (DLMF 10.51.2) and P_n' from the differentiated recurrence
//    T'_{n+1} = T_n + x T'_n - beta_n T'_{n-1};
//  * S' (target-normal derivative), n_t.grad_t: rho changes by that.n_t and
//    cos g by (1/rho)((d.n_t)/R - (that.n_t) cos g); j_n'(z) = (n/z) j_n -
//    j_{n+1} (DLMF 10.51.2); the 1/rho of the angular part multiplies
//    j_n(k rho), whose n = 1 term tends to k/3 as rho -> 0 (taken exactly).
// Summation: the g_n recurrence has real coefficients (2n+1)/z, so every sum
// sum_n c_n g_n with real c_n goes by Clenshaw's backward recurrence
// b_n = c_n + (2n+1)/z b_{n+1} - b_{n+2} (b_{p+1} = b_{p+2} = 0), sum =
// (c_0 - b_2) g_0 + b_1 g_1, in real arithmetic.  No g_n is formed beyond g_0
// and g_1, and the complex accumulation per order disappears.
//  * single layer: c_n = cj_n T_n;
//  * double layer: sum a_n (g_{n-1} - (n+1)/z g_n) = a_0/z + sum e_n g_n with
//    e_n = a_{n+1} - (n+1)/z a_n (g_{-1} = 1/z); its radial and angular
//    parts merge into one sequence c_n = (k a/R) e_n + u cj_n T'_n;
//  * S': c_n = (C/rho) cj_n T'_n + caj_n T_n, with the rho = 0 limit on g_1.
// T_n and T'_n go forward first and stay in registers.
// All of it -- Bessel and Hankel recurrences and the sums -- in FP64.
#include "helmholtz_items.cuh"

namespace tsqbx {

int launch_helmholtz_fp64(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const bool dlp = (layers & 2u) != 0;
    if (layers & 4u) return launch_helmholtz_fp64_sp(p, dlp, g, e, s);
    return dispatch_helm<false>(p, dlp, g, e, s, std::make_integer_sequence<int, 21>{});
}

}  // namespace tsqbx
