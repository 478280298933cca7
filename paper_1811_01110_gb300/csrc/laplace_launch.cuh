// laplace_launch.cuh -- the one-plan Laplace kernels (one warp per work item)
// and their dispatch over the expansion order p.  Each translation unit
// instantiates the variants it owns: laplace_fp64.cu / laplace_mixed.cu the
// single/double-layer ones, laplace_fp64_sp.cu / laplace_mixed_sp.cu the ones
// that also form S' (the target-normal derivative), so the four compile in
// parallel.  Besides one kernel per order p, each owns the runtime-order
// kernels (DevGeom::p_unroll 1, 2, 4; launch_runtime_order).
#pragma once

#include <utility>

#include "laplace_items.cuh"

namespace tsqbx {
namespace {

// Rows of a warp's staging tile (elements of `tile` sources each) and the
// dynamic shared memory of one CTA at staging depth `tile`.
template <bool MIXED, bool DLP>
__host__ __device__ constexpr int tile_rows() { return MIXED ? mixed_tile_rows(DLP) : (DLP ? 7 : 4); }
template <bool MIXED, bool DLP>
inline size_t tile_smem_bytes(int tile)
{
    // FP64: doubles per source; mixed: one 16-byte record per two sources
    return (size_t)kWarpsPerBlock * tile_rows<MIXED, DLP>() * (size_t)(MIXED ? (tile / 2) * 16 : tile * 8);
}

template <int P, bool DLP, bool SP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_fp64_kernel(const DevGeom g, const DevEval ev)
{
    extern __shared__ __align__(16) double smem_fp64[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;                       // whole warp leaves together
    double *T = smem_fp64 + (size_t)warp * tile_rows<false, DLP>() * g.tile;
    laplace_fp64_item<P, DLP, SP>(g, ev, g.items[item], g.item_walk[item], T, g.tile, lane);
}

template <int P, bool DLP, bool SP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
laplace_mixed_kernel(const DevGeom g, const DevEval ev)
{
    extern __shared__ __align__(16) float4 smem_mixed[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    if (item >= g.n_items) return;
    float4 *T = smem_mixed + (size_t)warp * tile_rows<true, DLP>() * (g.tile / 2);
    laplace_mixed_item<P, DLP, SP>(g, ev, g.items[item], g.item_walk[item], T, g.tile, lane);
}

template <bool MIXED, int P, bool DLP, bool SP>
void launch_one(unsigned blocks, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    static_assert((size_t)kWarpsPerBlock * tile_rows<MIXED, DLP>() * (MIXED ? (kTileMax / 2) * 16 : kTileMax * 8) <=
                      kSmemNoOptIn,
                  "staging tiles fit the default shared memory");
    const size_t smem = tile_smem_bytes<MIXED, DLP>(g.tile);
    if constexpr (MIXED) laplace_mixed_kernel<P, DLP, SP><<<blocks, kWarpsPerBlock * 32, smem, s>>>(g, e);
    else                 laplace_fp64_kernel<P, DLP, SP><<<blocks, kWarpsPerBlock * 32, smem, s>>>(g, e);
}

template <bool MIXED, bool SP, int P>
int launch_p(bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    if (!tile_depth_ok(g.tile)) return (int)cudaErrorInvalidValue;
    if (dlp) launch_one<MIXED, P, true, SP>((unsigned)blocks, g, e, s);
    else     launch_one<MIXED, P, false, SP>((unsigned)blocks, g, e, s);
    return (int)cudaGetLastError();
}

// The runtime-order kernels (DevGeom::p_unroll = 1, 2 or 4: one kernel for
// every order, its loop over n unrolled by that factor); the order is e.p.
template <bool MIXED, bool SP>
int launch_runtime_order(int unroll, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (e.p < 0 || e.p > kPMax) return (int)cudaErrorInvalidValue;
    const int64_t blocks = (g.n_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return 0;
    if (!tile_depth_ok(g.tile)) return (int)cudaErrorInvalidValue;
    const unsigned b = (unsigned)blocks;
    switch (unroll) {
    case 1: dlp ? launch_one<MIXED, -1, true, SP>(b, g, e, s) : launch_one<MIXED, -1, false, SP>(b, g, e, s); break;
    case 2: dlp ? launch_one<MIXED, -2, true, SP>(b, g, e, s) : launch_one<MIXED, -2, false, SP>(b, g, e, s); break;
    case 4: dlp ? launch_one<MIXED, -4, true, SP>(b, g, e, s) : launch_one<MIXED, -4, false, SP>(b, g, e, s); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

template <bool MIXED, bool SP, int... Ps>
int dispatch_p(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s,
               std::integer_sequence<int, Ps...>)
{
    int rc = (int)cudaErrorInvalidValue;
    ((p == Ps ? (rc = launch_p<MIXED, SP, Ps>(dlp, g, e, s), 0) : 0), ...);
    return rc;
}

// p in [0, 20]; any other p returns cudaErrorInvalidValue.  With
// g.p_unroll > 0 the runtime-order kernel runs (e.p must equal p).
template <bool MIXED, bool SP>
int laplace_dispatch(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s)
{
    if (g.p_unroll > 0) {
        if (e.p != p) return (int)cudaErrorInvalidValue;
        return launch_runtime_order<MIXED, SP>(g.p_unroll, dlp, g, e, s);
    }
    return dispatch_p<MIXED, SP>(p, dlp, g, e, s, std::make_integer_sequence<int, kPMax + 1>{});
}

}  // namespace

// Defined in laplace_fp64_sp.cu / laplace_mixed_sp.cu.
int launch_laplace_fp64_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s);
int launch_laplace_mixed_sp(int p, bool dlp, const DevGeom &g, const DevEval &e, cudaStream_t s);

}  // namespace tsqbx
