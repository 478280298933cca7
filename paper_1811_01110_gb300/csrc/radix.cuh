// radix.cuh -- two device primitives of the octree builder (octree.cu): an
// exclusive prefix sum of int arrays and a stable least-significant-digit
// radix sort of (int key, int value) pairs.  Both are exact integer
// computations, so their results do not depend on the launch shape.
//
// Scan: blocks of 1024 elements scanned by warp shuffles, the block totals
// scanned by one block in chunks, then added back.
//
// Sort: 8-bit digits, one pass per digit from the least significant.  A pass
// splits the input into tiles of kSortTile elements; each tile counts its
// digits (hist_kernel) into a digit-major table hist[digit * n_tiles + tile],
// whose exclusive prefix sum is where each (digit, tile) run starts in the
// output; scatter_kernel then writes every element to its run start plus the
// number of elements before it in the tile with the same digit.  Elements of
// a tile are taken in index order (round r, thread t: index r * 256 + t), and
// the rank counts equal digits in earlier rounds, in earlier warps of the
// round and in lower lanes of the warp (__match_any_sync), so equal keys
// keep their input order in every pass and the sort is stable.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace tsqbx {
namespace radix {
namespace {

constexpr int kScanBlock = 1024;                 // elements per scan block (one per thread)
constexpr int kSortThreads = 256;                // threads of a sort tile = digits per pass
constexpr int kSortItems = 4;                    // rounds per tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

// Inclusive prefix sum over the 1024 threads of a block; `total` receives the
// block's sum.  Every thread of the block must call it.
__device__ __forceinline__ int block_inclusive_scan(int v, int &total)
{
    __shared__ int warp_sum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += u;
    }
    if (lane == 31) warp_sum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sum[lane];                  // 32 warps of 32 threads
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += u;
        }
        warp_sum[lane] = w;                      // inclusive over warps
    }
    __syncthreads();
    total = warp_sum[31];
    const int before = warp > 0 ? warp_sum[warp - 1] : 0;
    __syncthreads();                             // warp_sum is reused by the next call
    return v + before;
}

// out[i] = sum of in[j], j < i, within each block of kScanBlock elements;
// block_sums[b] = the block's total.
__global__ void __launch_bounds__(kScanBlock) scan_blocks(const int *in, int *out, int64_t n, int *block_sums)
{
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int total;
    const int inc = block_inclusive_scan(v, total);
    if (i < n) out[i] = inc - v;
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Exclusive prefix sum of sums[0, nb) in place, by one block of kScanBlock
// threads in chunks (the running total carried across chunks).
__global__ void __launch_bounds__(kScanBlock) scan_sums(int *sums, int nb)
{
    int carry = 0;
    for (int base = 0; base < nb; base += kScanBlock) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? sums[i] : 0;
        int total;
        const int inc = block_inclusive_scan(v, total);
        if (i < nb) sums[i] = carry + inc - v;
        carry += total;
    }
}

__global__ void scan_add(int *out, int64_t n, const int *sums)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanBlock];
}

// Scratch ints exclusive_scan needs for n elements.
inline int64_t scan_scratch(int64_t n) { return (n + kScanBlock - 1) / kScanBlock; }

// out[i] = sum of in[j], j < i (exclusive).  scratch holds scan_scratch(n)
// ints.  Returns a cudaError_t.
inline cudaError_t exclusive_scan(const int *in, int *out, int64_t n, int *scratch, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = scan_scratch(n);
    scan_blocks<<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, n, scratch);
    scan_sums<<<1, kScanBlock, 0, s>>>(scratch, (int)nb);
    scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, scratch);
    return cudaGetLastError();
}

// Digit counts of one tile: hist[d * n_tiles + tile].
__global__ void __launch_bounds__(kSortThreads) hist_kernel(const int *key, int64_t n, int shift, int *hist,
                                                            int n_tiles)
{
    __shared__ int h[kSortThreads];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[((unsigned)key[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// One stable pass: element i of tile b with digit d goes to off[d * n_tiles +
// b] plus the number of equal digits before it in the tile.
__global__ void __launch_bounds__(kSortThreads) scatter_kernel(const int *key, const int *val, int64_t n, int shift,
                                                               const int *off, int n_tiles, int *key_out,
                                                               int *val_out)
{
    static_assert(kSortThreads == 256, "one thread per digit");
    __shared__ int run[kSortThreads];                  // next output position per digit
    __shared__ int wcount[kSortWarps][kSortThreads];   // this round's digit counts per warp
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    run[t] = off[(int64_t)t * n_tiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wcount[w][t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned below = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + r * kSortThreads + t;
        const bool valid = i < n;
        const int k = valid ? key[i] : 0;
        const int v = valid ? val[i] : 0;
        const int d = valid ? (int)(((unsigned)k >> shift) & 255u) : -1;   // -1: past the end
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & below);
        if (valid && rank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcount[w][d];
            key_out[pos] = k;
            val_out[pos] = v;
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            tot += wcount[w][t];
            wcount[w][t] = 0;
        }
        run[t] += tot;
        __syncthreads();
    }
}

// Scratch ints sort_pairs needs for n elements: two digit tables and the
// scan's block sums.
inline int64_t sort_scratch(int64_t n)
{
    const int64_t cells = (int64_t)kSortThreads * ((n + kSortTile - 1) / kSortTile);
    return 2 * cells + scan_scratch(cells);
}

// Stable sort of (key, val) pairs by the low `bits` bits of the keys
// (non-negative keys below 2^bits).  The pairs ping-pong between (key_a,
// val_a) and (key_b, val_b); *in_b tells where the sorted pairs are.
// scratch holds sort_scratch(n) ints.  Returns a cudaError_t.
inline cudaError_t sort_pairs(int *key_a, int *val_a, int *key_b, int *val_b, int64_t n, int bits, int *scratch,
                              bool *in_b, cudaStream_t s)
{
    *in_b = false;
    if (n <= 0) return cudaSuccess;
    const int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
    const int64_t cells = (int64_t)kSortThreads * n_tiles;
    int *hist = scratch, *off = scratch + cells, *sums = scratch + 2 * cells;
    int *k_in = key_a, *v_in = val_a, *k_out = key_b, *v_out = val_b;
    for (int shift = 0; shift < bits; shift += 8) {
        hist_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(k_in, n, shift, hist, (int)n_tiles);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = exclusive_scan(hist, off, cells, sums, s);
        if (e != cudaSuccess) return e;
        scatter_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(k_in, v_in, n, shift, off, (int)n_tiles, k_out,
                                                                  v_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        int *tk = k_in, *tv = v_in;
        k_in = k_out; v_in = v_out;
        k_out = tk; v_out = tv;
        *in_b = !*in_b;
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace radix
}  // namespace tsqbx
