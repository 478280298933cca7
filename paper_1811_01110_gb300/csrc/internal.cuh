// internal.cuh -- device-side layout shared by the libtsqbx kernels and the
// host plan code.  Not part of the public ABI (include/tsqbx.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tsqbx {

// Warp work item: the targets [slot_begin, slot_begin + n_tgt) of one group
// (all sharing that group's source list), L lanes per target, over the slice
// [src_lo, src_hi) of the group's source list (list positions).  part < 0: the item
// owns the whole list and writes the outputs; part >= 0: it writes partial
// sums to partial[part + j] (j < n_tgt), combined later in slice order.
struct __align__(16) Item {
    int32_t group, slot_begin, n_tgt, L;
    int32_t src_lo, src_hi, part, pad;
};

// Combine record: the targets [slot_begin, slot_begin + n_tgt) whose list was
// cut into n_slices slices; slice k's partials start at part + k * n_tgt.
struct __align__(16) Combine {
    int32_t slot_begin, n_tgt, part, n_slices;
};

constexpr int kWarpsPerBlock = 4;   // independent warps per CTA
// Sources staged per warp per shared-memory tile: kTile by default; a plan's
// tuning may choose any power of two in [kTileMin, kTileMax] (DevGeom::tile).
constexpr int kTile = 64;
constexpr int kTileMin = 32, kTileMax = 128;
// Shared memory a block may take without opting in to more: every kernel's
// staging tiles at the deepest depth stay within it (static_asserts beside
// each launch), so no launch needs cudaFuncSetAttribute.
constexpr size_t kSmemNoOptIn = 48 * 1024;
__host__ __device__ constexpr bool tile_depth_ok(int t)
{
    return t == 32 || t == 64 || t == 128;
}
constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;  // 1/(4 pi)

// Conventional-path records.  A center on the conventional path owns the
// target slots [slot_begin, slot_begin + n_tgt) (contiguous) and n_slices
// blocks of partial coefficients starting at block part0, one per
// coefficient-formation item (ConvItem) over its group's list.
struct __align__(16) ConvCenter {
    int32_t group, slot_begin, n_tgt, part0, n_slices, pad0, pad1, pad2;
};
struct __align__(16) ConvItem {              // P2QBXL: one center, one source slice
    int32_t center, src_lo, src_hi, part;
};
struct __align__(16) ConvEvalItem {          // QBXL2P: one center, <= 32 of its targets
    int32_t center, slot_begin, n_tgt, pad;
};

// Where an item's slice [src_lo, src_hi) of its group's list starts: run r,
// which covers the positions [p0, p1) and starts at source s0.  Computed once
// per schedule on the device, so an item's first sources load straight after
// the item record.
struct __align__(16) WalkStart {
    int32_t r, p0, p1, s0;
};

// Everything a kernel needs about a plan's geometry (device pointers).
struct DevGeom {
    int64_t n_src = 0, n_tgt = 0, n_items = 0, n_combine = 0, n_parts = 0;
    int32_t tile = kTile;               // staging depth of the one-plan kernels (tile_depth_ok)
    int32_t p_unroll = 0;               // Laplace FP64/mixed: 0 = per-order kernels, else the
                                        // runtime-order kernel with its loop unrolled by this
    int32_t fp64_share = 0;             // Laplace df64: items with (index mod 20) below this run
                                        // in native FP64 on the FP64 pipe (0..20)
    const Item *items = nullptr;
    const Combine *combine = nullptr;
    // Each group's source list as merged runs of consecutive sources: run r
    // (grp_run[q] <= r < grp_run[q+1]) holds the list positions up to
    // run_end[r] (exclusive; the group's previous run, or 0, gives its first)
    // and the sources run_src[r], run_src[r] + 1, ...  See ListWalk.
    const int64_t *grp_off = nullptr;   // [n_group+1] prefix sums of the list lengths
    const int32_t *grp_run = nullptr;   // [n_group+1] offsets into the run arrays
    const int32_t *run_end = nullptr;   // [n_runs] end of each run, as a list position
    const int32_t *run_src = nullptr;   // [n_runs] first source of each run
    int32_t n_runs = 0;
    const WalkStart *item_walk = nullptr;  // [n_items] where each item's slice starts
    // FP64 source records
    const double4_32a *src_pw = nullptr;    // {x, y, z, w}
    const double4_32a *src_n = nullptr;     // {nx, ny, nz, 0}
    // mixed-precision source records: coordinates as float-float pairs
    const float4 *src_hi = nullptr;     // {xh, yh, zh, 0}
    const float4 *src_lo = nullptr;     // {xl, yl, zl, 0}
    const float4 *src_nf = nullptr;     // {-nx, -ny, -nz, 0}: the negated normal
    // target slots, in item order
    const int32_t *slot_tgt = nullptr;  // output index of the slot's target
    const double4_32a *slot_c = nullptr;    // {cx, cy, cz, 0}
    const double4_32a *slot_e = nullptr;    // {ex, ey, ez, rho^2},  e = t - c
    const float4 *slot_chi = nullptr;   // float-float center
    const float4 *slot_clo = nullptr;
    const float4 *slot_ef = nullptr;    // {ex, ey, ez, -rho^2} rounded to FP32
    const double4_32a *slot_n = nullptr;    // target normal {nx, ny, nz, 0} (S')
    const float4 *slot_nf = nullptr;    // {n_t, -e.n_t} rounded to FP32 (mixed S')
    // conventional path
    int64_t n_conv_centers = 0, n_conv_items = 0, n_conv_eval = 0;
    const ConvCenter *conv_centers = nullptr;
    const ConvItem *conv_items = nullptr;
    const ConvEvalItem *conv_eval = nullptr;
};

// Source index at position k of one group's list, for positions that never
// decrease from one call to the next (each lane walks its own positions).
// Moving to the next run costs two loads from the small run arrays, which
// stay in cache; the list itself is never stored one entry per source.
// Positions must lie in the group's list; the walk never leaves the run arrays.
struct ListWalk {
    const int32_t *src, *end;
    int r, p0, p1, s0, r_last;
    __device__ __forceinline__ ListWalk(const DevGeom &g, const WalkStart &w)
        : src(g.run_src), end(g.run_end), r(w.r), p0(w.p0), p1(w.p1), s0(w.s0), r_last(g.n_runs - 1)
    {
    }
    // from the start of the group's list
    __device__ __forceinline__ ListWalk(const DevGeom &g, int group)
        : src(g.run_src), end(g.run_end), r(g.grp_run[group]), p0(0), r_last(g.n_runs - 1)
    {
        if (r < g.grp_run[group + 1]) {
            s0 = src[r];
            p1 = end[r];
        } else {
            s0 = 0;
            p1 = 0;
        }
    }
    __device__ __forceinline__ int at(int k)
    {
        while (k >= p1 && r < r_last) {
            ++r;
            p0 = p1;
            s0 = src[r];
            p1 = end[r];
        }
        return s0 + (k - p0);
    }
};

// The WalkStart of an item: the run of its group's list that holds position
// src_lo (a scan from the group's first run; an empty list gives p1 = 0).
__device__ __forceinline__ WalkStart walk_start_of(const DevGeom &g, const Item &it)
{
    int r = g.grp_run[it.group];
    const int r_end = g.grp_run[it.group + 1];
    if (r >= r_end) return WalkStart{r, 0, 0, 0};
    int p0 = 0, p1 = g.run_end[r];
    while (it.src_lo >= p1 && r + 1 < r_end) {
        p0 = p1;
        ++r;
        p1 = g.run_end[r];
    }
    return WalkStart{r, p0, p1, g.run_src[r]};
}

// Highest expansion order (TSQBX_P_MAX in tsqbx.h; plan.cu checks that they agree).
constexpr int kPMax = 20;
// Most densities one evaluation may carry (tsqbx_submit_multi_layers).
constexpr int kMaxRhs = 4;

// Per-evaluation buffers (device pointers).
struct DevEval {
    const double *wmu = nullptr;        // Laplace FP64: w_s mu_s
    const float *wmu_f = nullptr;       // Laplace mixed: (float)(w_s mu_s)
    const double2 *wmu_c = nullptr;     // Helmholtz: w_s mu_s (complex)
    double *out_slp = nullptr;          // indexed by target (real or interleaved complex)
    double *out_dlp = nullptr;
    double *out_sp = nullptr;
    double *part_slp = nullptr;         // partial sums of sliced items (scratch)
    double *part_dlp = nullptr;
    double *part_sp = nullptr;
    int *status = nullptr;              // bit 0: out-of-range source index seen
    double k = 0.0;                     // Helmholtz wavenumber
    int p = 0;                          // the evaluation's order (read by the runtime-order kernels)
    double *conv_coef = nullptr;        // conventional partial coefficients (scratch)
    // Several densities in one evaluation (the single layer of Helmholtz; the
    // single and double layers of Laplace in FP64 or double-float): the w mu
    // of density r starts at wmu_c (Helmholtz) or wmu (Laplace) + r *
    // rhs_src_stride, its outputs at out_rhs[r] / out_rhs_dlp[r] (NULL: layer
    // not formed) and its partial sums at part_slp / part_dlp + r *
    // rhs_part_stride (doubles).
    int n_rhs = 1;
    int64_t rhs_src_stride = 0;
    int64_t rhs_part_stride = 0;
    double *out_rhs[kMaxRhs] = {nullptr, nullptr, nullptr, nullptr};
    double *out_rhs_dlp[kMaxRhs] = {nullptr, nullptr, nullptr, nullptr};
};

// Launchers (one per translation unit).  Return a cudaError_t as int.
// Layer mask as in tsqbx.h (1 = single layer, 2 = double layer, 4 = S').
int launch_laplace_fp64(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_laplace_mixed(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_laplace_df64(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_helmholtz_fp64(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
// e.n_rhs (2..kMaxRhs) densities at once: the Helmholtz single layer; the
// Laplace single layer, or single and double layer (dlp), in FP64
// (laplace_multi.cu) and double-float (laplace_df64_multi.cu).
int launch_helmholtz_multi(int p, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_laplace_fp64_multi(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_laplace_df64_multi(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s);
// Conventional path: coefficient formation, then evaluation (Laplace in
// conventional.cu, Helmholtz in conventional_helm.cu).
int launch_conventional(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_conventional_helm(int p, unsigned layers, const DevGeom &g, const DevEval &e, cudaStream_t s);
// Orders the Helmholtz conventional path is compiled for (its unrolled complex
// triangles make higher orders slow to compile; the paper's Helmholtz
// computations use p <= 12).
constexpr int kConvHelmMaxP = 12;
// Doubles of one block of partial coefficients: (p+1)^2 real parts per layer
// formed (single layer when the mask has SLP or SP, double layer when it has
// DLP), twice that for the complex Helmholtz coefficients.
inline int conv_coef_doubles(int p, unsigned layers, bool helmholtz)
{
    return (helmholtz ? 2 : 1) * (p + 1) * (p + 1) * (((layers & 5u) ? 1 : 0) + ((layers & 2u) ? 1 : 0));
}

// Legendre three-term recurrence in the scaled form used by every kernel:
//   Q_n = (rho/R)^n P_n(x) = kappa_n T_n,
//   T_{n+1} = qx T_n - beta_n q2 T_{n-1},  qx = (rho/R) x,  q2 = (rho/R)^2,
// from Bonnet's (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1} with
// kappa_{n+1} = kappa_n (2n+1)/(n+1) and beta_n = n^2 / ((2n+1)(2n-1)).
__host__ __device__ constexpr double rec_kappa(int n)
{
    double k = 1.0;
    for (int m = 0; m < n; ++m) k *= (2.0 * m + 1.0) / (m + 1.0);
    return k;
}
__host__ __device__ constexpr double rec_beta(int n)
{
    return (1.0 * n * n) / ((2.0 * n + 1.0) * (2.0 * n - 1.0));
}

// The same for the derivatives alone.  With Q'_n = (rho/R)^{n-1} P_n'(x), the
// Legendre identities P'_{n+1} - x P'_n = (n+1) P_n and P'_{n+1} - P'_{n-1} =
// (2n+1) P_n give n Q'_{n+1} = (2n+1) qx Q'_n - (n+1) q2 Q'_{n-1} (the
// Gegenbauer C^(3/2) recurrence); scaled, Q'_n = lambda_n U_n,
//   U_{n+1} = qx U_n - gamma_n q2 U_{n-1},  U_0 = 0, U_1 = 1,
// lambda_{n+1} = lambda_n (2n+1)/n, lambda_1 = 1, gamma_n = (n^2-1)/(4n^2-1).
__host__ __device__ constexpr double rec_lambda(int n)
{
    double l = 1.0;
    for (int m = 1; m < n; ++m) l *= (2.0 * m + 1.0) / m;
    return l;
}
__host__ __device__ constexpr double rec_gamma(int n)
{
    return (1.0 * n * n - 1.0) / (4.0 * n * n - 1.0);
}

}  // namespace tsqbx
