// octree.cu -- the GIGAQBX octree and the near-field pair lists, built on the
// GPU (Sec. 3.1 and 3.2, Defs. 1-9: the tree over sources and QBX centers,
// colleagues, Lists 1-4 and their "close" variants under the target
// confinement region; the list building of Alg. 1 Stage 1).  The result is
// the List 1 + List 3 close + List 4 close source ranges of every box that
// owns a QBX center: the pair lists the TSQBX step takes.
//
// Rules (identical to the host builder of the input tooling, so the two can
// be compared bit for bit):
//  * root: the smallest power-of-two half width H with room for every source
//    and every QBX ball, center on the grid of spacing H/1024;
//  * a box owning more than n_max sources + centers splits: every source moves
//    to the child of its octant (p >= center per axis); a center moves only
//    if its ball fits in that child's target confinement region, radius
//    sqrt(3) h_child (1 + t_f); children receiving nothing are not created;
//    a box from which nothing moves stays a leaf;
//  * boxes are numbered breadth first, children in octant order; sources are
//    ordered depth first (each box's sources contiguous), a leaf's sources in
//    input order;
//  * two boxes are adjacent when the closed boxes intersect; a < TCR(b): the
//    center of a is at l2 distance >= 3|a| outside the TCR ball of b; TCR(a)
//    < b: the l-infinity distance from a's center to box b is >= 3|a|(1+t_f);
//  * List 1: leaves adjacent to the target box; List 3: descendants of the
//    colleagues' children not adjacent to it, closed under "a < TCR(b)"
//    (List 3 close: those that fail the test or hold fewer than n_mpole
//    sources); List 4: leaves coarser than the box adjacent to its parent but
//    not to it, and non-adjacent colleague leaves, gathered over the box and
//    its ancestors (List 4 close: those with TCR(box) < them false).
// Every floating-point test rounds each product and sum separately (explicit
// round-to-nearest intrinsics, no contraction), as the host builder does.
//
// Mapping: the tree is built level by level (one pass per level: count, mark
// the octants that receive points, prefix-sum the new boxes, move points);
// subtree source counts bottom up, depth-first offsets top down, and one
// stable radix sort of the sources by their leaf's offset (the prefix sums
// and the sort are this library's own, radix.cuh).  The lists use one
// thread per target box walking the tree with an explicit stack, in two
// passes (count, fill), then a per-box sort and merge of the ranges.
#include <algorithm>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <vector>

#include "internal.cuh"
#include "plan_internal.h"
#include "radix.cuh"
#include "tsqbx.h"

namespace tsqbx {
namespace {

constexpr int kMaxLevel = 30;       // deeper trees are rejected (coincident points)
constexpr int kStack = 256;         // >= 7 * kMaxLevel + 8 pending boxes

struct TreeView {
    int nb;
    const int *level, *parent, *child, *nsrc, *sbeg, *send;
    const char *leaf;
    const double *cx, *cy, *cz, *h;
    double t_f;
    int n_mpole;
};

__device__ __forceinline__ double cc(const TreeView &T, int k, int b) { return k == 0 ? T.cx[b] : k == 1 ? T.cy[b] : T.cz[b]; }

__device__ bool adjacent(const TreeView &T, int a, int b)
{
    for (int k = 0; k < 3; ++k)
        if (fabs(cc(T, k, a) - cc(T, k, b)) > T.h[a] + T.h[b]) return false;
    return true;
}

__device__ bool colleague2(const TreeView &T, int d, int b)
{
    for (int k = 0; k < 3; ++k)
        if (fabs(cc(T, k, d) - cc(T, k, b)) > 4.0 * T.h[b]) return false;
    return true;
}

__device__ double tcr_radius(const TreeView &T, int b)
{
    return __dmul_rn(__dmul_rn(sqrt(3.0), T.h[b]), __dadd_rn(1.0, T.t_f));
}

// a < TCR(b)
__device__ bool sep_box_tcr(const TreeView &T, int a, int b)
{
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double t = __dsub_rn(cc(T, k, a), cc(T, k, b));
        d2 = __dadd_rn(d2, __dmul_rn(t, t));
    }
    return __dsub_rn(__dsqrt_rn(d2), tcr_radius(T, b)) >= __dmul_rn(3.0, T.h[a]);
}

// TCR(a) < b (l-infinity sufficient check)
__device__ bool sep_tcr_box(const TreeView &T, int a, int b)
{
    double dist = 0.0;
    for (int k = 0; k < 3; ++k) dist = fmax(dist, __dsub_rn(fabs(__dsub_rn(cc(T, k, a), cc(T, k, b))), T.h[b]));
    return dist >= __dmul_rn(__dmul_rn(3.0, T.h[a]), __dadd_rn(1.0, T.t_f));
}

// Same-level 2-colleagues of b (b included), by a pruned descent.
__device__ int colleagues(const TreeView &T, int b, int *out)
{
    int stack[kStack], sp = 0, n = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const int x = stack[--sp];
        bool far = false;
        for (int k = 0; k < 3; ++k)
            if (fabs(cc(T, k, x) - cc(T, k, b)) > T.h[x] + 5.0 * T.h[b]) far = true;
        if (far) continue;
        if (T.level[x] == T.level[b]) {
            if (colleague2(T, x, b) && n < 128) out[n++] = x;
            continue;
        }
        for (int o = 7; o >= 0; --o) {
            const int c = T.child[8 * x + o];
            if (c >= 0 && sp < kStack) stack[sp++] = c;
        }
    }
    return n;
}

// Raw List 4 of box a (a target box or an ancestor of one): leaves coarser
// than a, adjacent to parent(a) but not to a, and a's non-adjacent colleague
// leaves (coll: a's colleagues); emit(d) for each.
template <class Emit>
__device__ void raw_list4(const TreeView &T, int a, const int *coll, int nc, Emit &emit)
{
    const int pa = T.parent[a];
    if (pa >= 0) {
        int stack[kStack], sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const int x = stack[--sp];
            if (T.level[x] >= T.level[a] || !adjacent(T, x, pa)) continue;
            if (T.leaf[x]) {
                if (T.nsrc[x] > 0 && !adjacent(T, x, a)) emit(x);
                continue;
            }
            for (int o = 7; o >= 0; --o) {
                const int c = T.child[8 * x + o];
                if (c >= 0 && sp < kStack) stack[sp++] = c;
            }
        }
    }
    for (int i = 0; i < nc; ++i) {
        const int d = coll[i];
        if (T.leaf[d] && T.nsrc[d] > 0 && !adjacent(T, d, a)) emit(d);
    }
}

// CSR lists per "list box" (target boxes and their ancestors): colleagues
// and raw List 4; pos[b] = the box's row, -1 if it has none.
struct BoxLists {
    const int *pos;
    const long long *coll_off;
    const int *coll;
    const long long *l4_off;
    const int *l4;
};

struct CountEmit {
    int n = 0;
    __device__ void operator()(int) { ++n; }
};
struct BoxEmit {
    int *out;
    int n = 0;
    __device__ void operator()(int b) { out[n++] = b; }
};

// Colleagues of each list box (count or fill).
template <bool FILL>
__global__ void coll_kernel(const TreeView T, const int *boxes, int n, const long long *off, int *out, int *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[128];
    const int m = colleagues(T, boxes[i], c);
    if (FILL) for (int k = 0; k < m; ++k) out[off[i] + k] = c[k];
    else count[i] = m;
}

// Raw List 4 of each list box (count or fill).
template <bool FILL>
__global__ void l4_kernel(const TreeView T, const int *boxes, int n, const long long *coll_off, const int *coll,
                          const long long *off, int *out, int *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nc = (int)(coll_off[i + 1] - coll_off[i]);
    if (FILL) {
        BoxEmit e{out + off[i]};
        raw_list4(T, boxes[i], coll + coll_off[i], nc, e);
    } else {
        CountEmit e;
        raw_list4(T, boxes[i], coll + coll_off[i], nc, e);
        count[i] = e.n;
    }
}

// Warp-cooperative near field of target box w: one shared stack of typed
// entries (box | mode << 29) holds the List 1 walk (from the root), the
// List 3 walks (from the colleagues' children) and the List 3 classification;
// each step the lanes pop up to 32 entries, process one each, and push their
// children at offsets from a warp prefix sum.  List 4 close is a lane-strided
// filter over the raw List 4 of w and its ancestors.  emit(lane, box) is
// called by the lane that found the box (any order: the ranges are sorted
// afterwards).  Returns false if the stack overflowed (never silently).
constexpr int kWarpStack = 4096;
constexpr int kNearWarps = 2;
enum : int { kModeL1 = 0, kModeL3 = 1, kModeCls = 2 };

template <class Emit>
__device__ bool near_field_warp(const TreeView &T, const BoxLists &BL, int w, int lane, int *stk, Emit &emit)
{
    int top = 0;
    bool ok = true;
    // initial entries: the root (List 1) and the colleagues' children (List 3)
    if (lane == 0) stk[0] = 0 | (kModeL1 << 29);
    top = 1;
    const int row = BL.pos[w];
    const long long c0 = BL.coll_off[row], c1 = BL.coll_off[row + 1];
    for (long long base = c0 * 8; base < c1 * 8; base += 32) {
        const long long j = base + lane;
        int c = -1;
        if (j < c1 * 8) c = T.child[8 * BL.coll[j / 8] + (int)(j % 8)];
        const unsigned m = __ballot_sync(0xffffffffu, c >= 0);
        const int pos = __popc(m & ((1u << lane) - 1));
        if (c >= 0) {
            if (top + pos < kWarpStack) stk[top + pos] = c | (kModeL3 << 29);
        }
        top += __popc(m);
        if (top > kWarpStack) ok = false;
    }
    __syncwarp();
    while (top > 0 && ok) {
        const int take = min(32, top);
        top -= take;
        const int e = lane < take ? stk[top + lane] : -1;
        __syncwarp();
        int kids[8], nk = 0, mode = 0;
        if (e >= 0) {
            const int x = e & ((1 << 29) - 1);
            mode = e >> 29;
            bool expand = false;
            if (mode == kModeL1) {
                if (adjacent(T, x, w)) {
                    if (T.leaf[x]) { if (T.nsrc[x] > 0) emit(lane, x); }
                    else expand = true;
                }
            } else if (T.nsrc[x] > 0) {
                if (mode == kModeL3 && adjacent(T, x, w)) {
                    expand = !T.leaf[x];
                } else {                       // a List 3 box, or below one: classify
                    mode = kModeCls;
                    if (sep_box_tcr(T, x, w)) { if (T.nsrc[x] < T.n_mpole) emit(lane, x); }
                    else if (T.leaf[x]) emit(lane, x);
                    else expand = true;
                }
            }
            if (expand)
                for (int o = 0; o < 8; ++o) {
                    const int c = T.child[8 * x + o];
                    if (c >= 0) kids[nk++] = c;
                }
        }
        // warp prefix sum of the pushes
        int incl = nk;
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (top + total > kWarpStack) { ok = false; break; }
        const int at = top + incl - nk;
        for (int i = 0; i < nk; ++i) stk[at + i] = kids[i] | (mode << 29);
        top += total;
        __syncwarp();
    }
    // List 4 close
    for (int a = w; a >= 0; a = T.parent[a]) {
        const int r = BL.pos[a];
        for (long long i = BL.l4_off[r] + lane; i < BL.l4_off[r + 1]; i += 32) {
            const int d = BL.l4[i];
            if (!sep_tcr_box(T, w, d)) emit(lane, d);
        }
    }
    __syncwarp();
    return ok;
}

struct WarpCount {
    int n = 0;
    __device__ void operator()(int, int) { ++n; }
};
struct WarpFill {
    const TreeView *T;
    int2 *out;
    int *cursor;             // shared per-warp append position
    __device__ void operator()(int, int b)
    {
        const int k = atomicAdd(cursor, 1);
        out[k] = make_int2(T->sbeg[b], T->send[b]);
    }
};

__global__ void __launch_bounds__(kNearWarps * 32)
near_count_kernel(const TreeView T, const BoxLists BL, const int *tboxes, int nt, int *count, int *status)
{
    __shared__ int stk_all[kNearWarps][kWarpStack];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kNearWarps + warp;
    if (i >= nt) return;
    WarpCount e;
    const bool ok = near_field_warp(T, BL, tboxes[i], lane, stk_all[warp], e);
    int n = e.n;
    for (int d = 16; d > 0; d >>= 1) n += __shfl_xor_sync(0xffffffffu, n, d);
    if (lane == 0) {
        count[i] = n;
        if (!ok) atomicOr(status, 1);
    }
}

// Ascending sort of a[0, P) by (x, y) in shared memory by one warp (bitonic
// network; P a power of two).  Equal ranges may change places, which the
// merge that follows cannot tell apart.
__device__ void bitonic_sort_warp(int2 *a, int P, int lane)
{
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < P / 2; t += 32) {
                const int i = 2 * t - (t & (j - 1));        // the t-th index with bit j clear
                const int l = i + j;
                const bool up = (i & k) == 0;
                const int2 x = a[i], y = a[l];
                const bool gt = x.x > y.x || (x.x == y.x && x.y > y.y);
                if (gt == up) {
                    a[i] = y;
                    a[l] = x;
                }
            }
            __syncwarp();
        }
}

__global__ void __launch_bounds__(kNearWarps * 32)
near_fill_kernel(const TreeView T, const BoxLists BL, const int *tboxes, int nt, const long long *off, int2 *raw,
                 int2 *sorted, int *merged, int *status)
{
    __shared__ __align__(16) int stk_all[kNearWarps][kWarpStack];
    __shared__ int cursor[kNearWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kNearWarps + warp;
    if (i >= nt) return;
    if (lane == 0) cursor[warp] = 0;
    __syncwarp();
    WarpFill e{&T, raw + off[i], &cursor[warp]};
    const bool ok = near_field_warp(T, BL, tboxes[i], lane, stk_all[warp], e);
    __syncwarp();
    if (lane == 0 && !ok) atomicOr(status, 1);
    // sort by (begin, end): chunks of up to kChunk ranges in the (now free)
    // stack by a bitonic network; with several chunks, each range then goes
    // to its index in its chunk plus the number of ranges before it in the
    // other chunks (binary searches; equal ranges of earlier chunks first)
    constexpr int kChunk = kWarpStack / 2;
    const int n = cursor[warp];
    int2 *r = raw + off[i];
    int2 *out = sorted + off[i];
    int2 *buf = reinterpret_cast<int2 *>(stk_all[warp]);
    for (int c0 = 0; c0 < n; c0 += kChunk) {
        const int m = min(kChunk, n - c0);
        int P = 1;
        while (P < m) P <<= 1;
        for (int k = lane; k < P; k += 32) buf[k] = k < m ? r[c0 + k] : make_int2(INT_MAX, INT_MAX);
        __syncwarp();
        bitonic_sort_warp(buf, P, lane);
        int2 *dst = n <= kChunk ? out : r;
        for (int k = lane; k < m; k += 32) dst[c0 + k] = buf[k];
        __syncwarp();
    }
    if (n > kChunk) {
        const int nch = (n + kChunk - 1) / kChunk;
        for (int k = lane; k < n; k += 32) {
            const int a = k / kChunk;
            const int2 v = r[k];
            int pos = k - a * kChunk;
            for (int b = 0; b < nch; ++b) {
                if (b == a) continue;
                const int lo0 = b * kChunk;
                int lo = lo0, hi = min(n, lo0 + kChunk);
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    const int2 u = r[mid];
                    const bool before = u.x < v.x || (u.x == v.x && (u.y < v.y || (u.y == v.y && b < a)));
                    if (before) lo = mid + 1;
                    else hi = mid;
                }
                pos += lo - lo0;
            }
            out[pos] = v;
        }
        __syncwarp();
    }
    if (lane != 0) return;
    // drop empty ranges and join touching ones (into raw)
    int2 *m_out = raw + off[i];
    int m = 0;
    for (int a = 0; a < n; ++a) {
        const int2 v = out[a];
        if (v.x == v.y) continue;
        if (m > 0 && m_out[m - 1].y == v.x) m_out[m - 1].y = v.y;
        else m_out[m++] = v;
    }
    merged[i] = m;
}

// Gathers each target box's merged ranges (the first merged[i] of its raw
// block at off[i]) into the contiguous near_begin / near_end arrays at moff[i];
// one warp per box.
__global__ void compact_near_kernel(const int2 *raw, const long long *off, const int *merged,
                                    const long long *moff, int nt, int *near_begin, int *near_end)
{
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nt; i += (gridDim.x * blockDim.x) >> 5) {
        const int2 *src = raw + off[i];
        const long long at = moff[i];
        for (int k = lane; k < merged[i]; k += 32) {
            const int2 v = src[k];
            near_begin[at + k] = v.x;
            near_end[at + k] = v.y;
        }
    }
}

// ------------------------------------------------------------- tree building

__global__ void bbox_kernel(int64_t ns, const double *s, int64_t nc, const double *c, const double *r,
                            double *part)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += stride)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], s[k * ns + i]);
            hi[k] = fmax(hi[k], s[k * ns + i]);
        }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += stride)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __dsub_rn(c[k * nc + i], r[i]));
            hi[k] = fmax(hi[k], __dadd_rn(c[k * nc + i], r[i]));
        }
    for (int k = 0; k < 3; ++k)
        for (int off = 16; off > 0; off >>= 1) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
        }
    __shared__ double sh[32][6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) { sh[warp][k] = lo[k]; sh[warp][3 + k] = hi[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 3; ++k) {
                sh[0][k] = fmin(sh[0][k], sh[w][k]);
                sh[0][3 + k] = fmax(sh[0][3 + k], sh[w][3 + k]);
            }
        for (int k = 0; k < 6; ++k) part[6 * blockIdx.x + k] = sh[0][k];
    }
}

struct BuildBuf {
    int *level, *parent, *child, *nsrc, *sbeg, *send, *nctr;
    char *leaf;
    double *cx, *cy, *cz, *h;
};

// Count the points of each box of the current level (boxes [lb, lb + nlev)).
// Few boxes (the top levels): counted in shared memory first, one global
// atomic per box and block.
constexpr int kSmemBoxes = 4096;
__global__ void count_kernel(int64_t ns, const int *sbox, const char *sact, int64_t nc, const int *cbox,
                             const char *cact, int lb, int nlev, int *cnt)
{
    __shared__ int sh[kSmemBoxes];
    const bool local = nlev <= kSmemBoxes;
    if (local) {
        for (int i = threadIdx.x; i < nlev; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    int *dst = local ? sh : cnt;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns + nc; i += stride) {
        if (i < ns) { if (sact[i]) atomicAdd(&dst[sbox[i] - lb], 1); }
        else { const int64_t j = i - ns; if (cact[j]) atomicAdd(&dst[cbox[j] - lb], 1); }
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < nlev; i += blockDim.x)
            if (sh[i]) atomicAdd(&cnt[i], sh[i]);
    }
}

// Octant of every active point of a splitting box; marks receiving octants.
// oct >= 0: moves there; -1: its box does not split (settles); -2: a center
// whose ball does not fit its octant's child (stays in the split box).
__global__ void octant_kernel(int64_t ns, const double *s, const int *sbox, const char *sact, int *soct,
                              int64_t nc, const double *c, const double *r, const int *cbox, const char *cact,
                              int *coct, BuildBuf B, int lb, const int *cnt, int n_max, double t_f, int *flag)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns + nc; i += stride) {
        const bool is_src = i < ns;
        const int64_t j = is_src ? i : i - ns;
        if (!(is_src ? sact[j] : cact[j])) continue;
        const int b = is_src ? sbox[j] : cbox[j];
        if (cnt[b - lb] <= n_max) { (is_src ? soct : coct)[j] = -1; continue; }
        const int64_t n = is_src ? ns : nc;
        const double *x = is_src ? s : c;
        const double p[3] = {x[j], x[n + j], x[2 * n + j]};
        const double bc[3] = {B.cx[b], B.cy[b], B.cz[b]};
        int o = 0;
        for (int k = 0; k < 3; ++k) if (p[k] >= bc[k]) o |= 1 << k;
        if (!is_src) {
            const double hh = 0.5 * B.h[b];
            const double rt = __dmul_rn(__dmul_rn(sqrt(3.0), hh), __dadd_rn(1.0, t_f));
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double kc = bc[k] + (((o >> k) & 1) ? hh : -hh);
                const double t = __dsub_rn(p[k], kc);
                d2 = __dadd_rn(d2, __dmul_rn(t, t));
            }
            if (!(__dadd_rn(__dsqrt_rn(d2), r[j]) <= rt)) { coct[j] = -2; continue; }
        }
        (is_src ? soct : coct)[j] = o;
        flag[8 * (b - lb) + o] = 1;
    }
}

__global__ void children_kernel(BuildBuf B, int lb, int nlev, const int *flag, const int *off, int le)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * nlev) return;
    if (!flag[i]) return;
    const int b = lb + i / 8, o = i % 8, id = le + off[i];
    const double hh = 0.5 * B.h[b];
    B.level[id] = B.level[b] + 1;
    B.h[id] = hh;
    B.cx[id] = B.cx[b] + ((o & 1) ? hh : -hh);
    B.cy[id] = B.cy[b] + ((o & 2) ? hh : -hh);
    B.cz[id] = B.cz[b] + ((o & 4) ? hh : -hh);
    B.parent[id] = b;
    for (int q = 0; q < 8; ++q) B.child[8 * id + q] = -1;
    B.leaf[id] = 1;
    B.child[8 * b + o] = id;
    B.leaf[b] = 0;
}

__global__ void move_kernel(int64_t ns, int *sbox, char *sact, const int *soct, int64_t nc, int *cbox, char *cact,
                            const int *coct, const int *child)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns + nc; i += stride) {
        if (i < ns) {
            if (!sact[i]) continue;
            if (soct[i] >= 0) sbox[i] = child[8 * sbox[i] + soct[i]];
            else sact[i] = 0;
        } else {
            const int64_t j = i - ns;
            if (!cact[j]) continue;
            if (coct[j] >= 0) cbox[j] = child[8 * cbox[j] + coct[j]];
            else cact[j] = 0;
        }
    }
}

__global__ void leaf_counts_kernel(int64_t ns, const int *sbox, int64_t nc, const int *cbox, int *nsrc, int *nctr)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns + nc; i += stride) {
        if (i < ns) atomicAdd(&nsrc[sbox[i]], 1);
        else atomicAdd(&nctr[cbox[i - ns]], 1);
    }
}

__global__ void up_kernel(const int *parent, int lb, int le, int *nsrc)
{
    const int b = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (b < le && nsrc[b] > 0) atomicAdd(&nsrc[parent[b]], nsrc[b]);
}

__global__ void down_kernel(const int *child, const int *nsrc, int lb, int le, int *sbeg, int *send)
{
    const int b = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= le) return;
    int run = sbeg[b];
    send[b] = run + nsrc[b];
    for (int o = 0; o < 8; ++o) {
        const int c = child[8 * b + o];
        if (c < 0) continue;
        sbeg[c] = run;
        run += nsrc[c];
    }
}

__global__ void sort_keys_kernel(int64_t ns, const int *sbox, const int *sbeg, int *key, int *val)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += stride) {
        key[i] = sbeg[sbox[i]];
        val[i] = (int)i;
    }
}

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    void alloc(size_t count)
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = count;
        if (count) {
            if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
        }
    }
    void grow(size_t count)     // keeps the contents
    {
        if (count <= n) return;
        T *q = nullptr;
        if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
        if (p) { cudaMemcpy(q, p, n * sizeof(T), cudaMemcpyDeviceToDevice); cudaFree(p); }
        p = q;
        n = count;
    }
    ~DBuf() { if (p) cudaFree(p); }
};

}  // namespace
}  // namespace tsqbx

using namespace tsqbx;

struct tsqbx_octree_s {
    int64_t n_src = 0, n_ctr = 0, n_boxes = 0;
    std::vector<int32_t> level, parent, src_begin, src_end, n_owned_ctr, is_leaf, src_perm, ctr_box;
    std::vector<double> center, halfwidth;
    std::vector<int64_t> near_start;
    std::vector<int32_t> near_begin, near_end;
    tsqbx_octree_stats stats{};
};

namespace {

bool finite_all(const double *x, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

int grid_for(int64_t n, int n_sm)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 8));
}

template <class T>
void to_host(std::vector<T> &v, const T *d, size_t n)
{
    v.resize(n);
    if (n) ck(cudaMemcpy(v.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost));
}

void build(tsqbx_octree_s &O, int64_t ns, const double *hs, int64_t nc, const double *hc, const double *hr,
           int n_max, double t_f, int n_mpole, int n_sm)
{
    using clk = std::chrono::steady_clock;
    auto t_mark = clk::now();
    auto lap = [&](double &dst) {
        ck(cudaDeviceSynchronize());
        const auto now = clk::now();
        dst = std::chrono::duration<double, std::milli>(now - t_mark).count();
        t_mark = now;
    };
    DBuf<double> s, c, r;
    s.alloc(3 * ns); c.alloc(3 * nc); r.alloc(nc);
    if (ns) ck(cudaMemcpy(s.p, hs, 3 * ns * sizeof(double), cudaMemcpyHostToDevice));
    if (nc) {
        ck(cudaMemcpy(c.p, hc, 3 * nc * sizeof(double), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(r.p, hr, nc * sizeof(double), cudaMemcpyHostToDevice));
    }
    const int64_t np = ns + nc;
    const int gp = grid_for(np, n_sm);
    lap(O.stats.upload_ms);

    // bounding cube of the sources and QBX balls; root as in the host builder
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    {
        DBuf<double> part;
        part.alloc(6 * (size_t)gp);
        bbox_kernel<<<gp, 256>>>(ns, s.p, nc, c.p, r.p, part.p);
        ck(cudaGetLastError());
        std::vector<double> h;
        to_host(h, part.p, 6 * (size_t)gp);
        for (int b = 0; b < gp; ++b)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], h[6 * b + k]);
                hi[k] = std::max(hi[k], h[6 * b + 3 + k]);
            }
    }
    double half = 0;
    for (int k = 0; k < 3; ++k) half = std::max(half, 0.5 * (hi[k] - lo[k]));
    double H = std::ldexp(1.0, (int)std::ceil(std::log2(std::max(half, 1e-30))));
    double q = H / 1024.0;
    if (half + q > H) { H *= 2.0; q *= 2.0; }
    double rootc[3];
    for (int k = 0; k < 3; ++k) rootc[k] = std::round(0.5 * (lo[k] + hi[k]) / q) * q;

    // boxes (grown as levels are added)
    DBuf<int> level, parent, child, nsrc, sbeg, send, nctr;
    DBuf<char> leaf;
    DBuf<double> cx, cy, cz, hw;
    size_t cap = 0;
    auto ensure = [&](size_t need) {
        if (need <= cap) return;
        size_t nc2 = std::max<size_t>(need, 2 * cap + 64);
        level.grow(nc2); parent.grow(nc2); child.grow(8 * nc2); leaf.grow(nc2);
        cx.grow(nc2); cy.grow(nc2); cz.grow(nc2); hw.grow(nc2);
        cap = nc2;
    };
    ensure(1);
    {
        const int zero = 0, m1 = -1;
        const char one = 1;
        ck(cudaMemcpy(level.p, &zero, sizeof(int), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(parent.p, &m1, sizeof(int), cudaMemcpyHostToDevice));
        std::vector<int> ch(8, -1);
        ck(cudaMemcpy(child.p, ch.data(), 8 * sizeof(int), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(leaf.p, &one, 1, cudaMemcpyHostToDevice));
        ck(cudaMemcpy(cx.p, &rootc[0], sizeof(double), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(cy.p, &rootc[1], sizeof(double), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(cz.p, &rootc[2], sizeof(double), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(hw.p, &H, sizeof(double), cudaMemcpyHostToDevice));
    }
    // points: current box, still moving, octant of this level
    DBuf<int> sbox, soct, cbox, coct;
    DBuf<char> sact, cact;
    sbox.alloc(ns); soct.alloc(ns); sact.alloc(ns); cbox.alloc(nc); coct.alloc(nc); cact.alloc(nc);
    if (ns) { ck(cudaMemset(sbox.p, 0, ns * sizeof(int))); ck(cudaMemset(sact.p, 1, ns)); }
    if (nc) { ck(cudaMemset(cbox.p, 0, nc * sizeof(int))); ck(cudaMemset(cact.p, 1, nc)); }

    std::vector<int> lev_begin{0};
    int lb = 0, le = 1;
    DBuf<int> cnt, flag, off;
    DBuf<int> tmp;                                      // scan and sort scratch
    while (lb < le) {
        if ((int)lev_begin.size() > kMaxLevel + 1) throw std::invalid_argument("octree too deep");
        const int nlev = le - lb;
        cnt.alloc(nlev); flag.alloc(8 * (size_t)nlev); off.alloc(8 * (size_t)nlev);
        ck(cudaMemset(cnt.p, 0, nlev * sizeof(int)));
        ck(cudaMemset(flag.p, 0, 8 * (size_t)nlev * sizeof(int)));
        count_kernel<<<gp, 256>>>(ns, sbox.p, sact.p, nc, cbox.p, cact.p, lb, nlev, cnt.p);
        ck(cudaGetLastError());
        BuildBuf B{level.p, parent.p, child.p, nullptr, nullptr, nullptr, nullptr, leaf.p, cx.p, cy.p, cz.p, hw.p};
        octant_kernel<<<gp, 256>>>(ns, s.p, sbox.p, sact.p, soct.p, nc, c.p, r.p, cbox.p, cact.p, coct.p, B, lb, cnt.p,
                                   n_max, t_f, flag.p);
        ck(cudaGetLastError());
        const int64_t n_flag = 8 * (int64_t)nlev;
        if ((size_t)radix::scan_scratch(n_flag) > tmp.n) tmp.alloc(radix::scan_scratch(n_flag));
        ck(radix::exclusive_scan(flag.p, off.p, n_flag, tmp.p, 0));
        int last[2] = {0, 0};
        ck(cudaMemcpy(&last[0], off.p + 8 * nlev - 1, sizeof(int), cudaMemcpyDeviceToHost));
        ck(cudaMemcpy(&last[1], flag.p + 8 * nlev - 1, sizeof(int), cudaMemcpyDeviceToHost));
        const int n_new = last[0] + last[1];
        ensure((size_t)le + n_new);
        B = BuildBuf{level.p, parent.p, child.p, nullptr, nullptr, nullptr, nullptr, leaf.p, cx.p, cy.p, cz.p, hw.p};
        if (n_new > 0) {
            children_kernel<<<(8 * nlev + 255) / 256, 256>>>(B, lb, nlev, flag.p, off.p, le);
            ck(cudaGetLastError());
        }
        move_kernel<<<gp, 256>>>(ns, sbox.p, sact.p, soct.p, nc, cbox.p, cact.p, coct.p, child.p);
        ck(cudaGetLastError());
        lb = le;
        le += n_new;
        lev_begin.push_back(lb);
    }
    const int nb = le;
    const int n_levels = (int)lev_begin.size() - 1;      // lev_begin[L] .. lev_begin[L+1]
    lap(O.stats.tree_ms);

    // subtree source counts (bottom up), depth-first offsets (top down)
    nsrc.alloc(nb); nctr.alloc(nb); sbeg.alloc(nb); send.alloc(nb);
    ck(cudaMemset(nsrc.p, 0, nb * sizeof(int)));
    ck(cudaMemset(nctr.p, 0, nb * sizeof(int)));
    ck(cudaMemset(sbeg.p, 0, nb * sizeof(int)));
    leaf_counts_kernel<<<gp, 256>>>(ns, sbox.p, nc, cbox.p, nsrc.p, nctr.p);
    ck(cudaGetLastError());
    for (int L = n_levels - 1; L >= 1; --L) {
        const int a = lev_begin[L], b = lev_begin[L + 1];
        up_kernel<<<(b - a + 255) / 256, 256>>>(parent.p, a, b, nsrc.p);
        ck(cudaGetLastError());
    }
    for (int L = 0; L < n_levels; ++L) {
        const int a = lev_begin[L], b = lev_begin[L + 1];
        down_kernel<<<(b - a + 255) / 256, 256>>>(child.p, nsrc.p, a, b, sbeg.p, send.p);
        ck(cudaGetLastError());
    }
    // depth-first source order: stable sort by the leaf's offset
    DBuf<int> key, val, key2, val2;
    key.alloc(ns); val.alloc(ns); key2.alloc(ns); val2.alloc(ns);
    const int *perm = val.p;                            // the sorted source indices
    if (ns) {
        sort_keys_kernel<<<grid_for(ns, n_sm), 256>>>(ns, sbox.p, sbeg.p, key.p, val.p);
        ck(cudaGetLastError());
        int bits = 1;
        while ((int64_t)1 << bits <= ns) ++bits;
        if ((size_t)radix::sort_scratch(ns) > tmp.n) tmp.alloc(radix::sort_scratch(ns));
        bool in_b = false;
        ck(radix::sort_pairs(key.p, val.p, key2.p, val2.p, ns, bits, tmp.p, &in_b, 0));
        perm = in_b ? val2.p : val.p;
    }

    lap(O.stats.order_ms);
    // near-field lists of the target boxes
    to_host(O.n_owned_ctr, nctr.p, nb);
    std::vector<int> par;
    to_host(par, parent.p, nb);
    std::vector<char> toa(nb, 0);                      // target box or ancestor of one
    std::vector<int> tboxes, lboxes, pos(nb, -1);
    for (int b = 0; b < nb; ++b) {
        if (O.n_owned_ctr[b] <= 0) continue;
        tboxes.push_back(b);
        for (int a = b; a >= 0 && !toa[a]; a = par[a]) toa[a] = 1;
    }
    for (int b = 0; b < nb; ++b)
        if (toa[b]) { pos[b] = (int)lboxes.size(); lboxes.push_back(b); }
    const int nt = (int)tboxes.size(), nl = (int)lboxes.size();
    TreeView T{nb, level.p, parent.p, child.p, nsrc.p, sbeg.p, send.p, leaf.p, cx.p, cy.p, cz.p, hw.p, t_f, n_mpole};
    std::vector<long long> hoff(nt + 1, 0);
    std::vector<int> hmerged(nt);
    DBuf<int2> raw;
    DBuf<int> near_b, near_e;
    long long n_near = 0;
    // CSR from per-row counts (prefix sum on the host: one copy each way)
    auto csr = [&](DBuf<int> &dcount, int n, DBuf<long long> &doff) {
        std::vector<int> hc;
        to_host(hc, dcount.p, n);
        std::vector<long long> o(n + 1, 0);
        for (int i = 0; i < n; ++i) o[i + 1] = o[i] + hc[i];
        doff.alloc(n + 1);
        ck(cudaMemcpy(doff.p, o.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice));
        return o;
    };
    if (nt > 0) {
        DBuf<int> dl, dpos, dcount, dcoll, dl4, dt;
        DBuf<long long> dcoll_off, dl4_off, doff;
        dl.alloc(nl); dpos.alloc(nb); dcount.alloc(std::max(nl, nt));
        ck(cudaMemcpy(dl.p, lboxes.data(), nl * sizeof(int), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(dpos.p, pos.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
        const int gl = (nl + 127) / 128;
        coll_kernel<false><<<gl, 128>>>(T, dl.p, nl, nullptr, nullptr, dcount.p);
        ck(cudaGetLastError());
        const std::vector<long long> co = csr(dcount, nl, dcoll_off);
        dcoll.alloc(std::max<long long>(1, co[nl]));
        coll_kernel<true><<<gl, 128>>>(T, dl.p, nl, dcoll_off.p, dcoll.p, nullptr);
        ck(cudaGetLastError());
        l4_kernel<false><<<gl, 128>>>(T, dl.p, nl, dcoll_off.p, dcoll.p, nullptr, nullptr, dcount.p);
        ck(cudaGetLastError());
        const std::vector<long long> lo4 = csr(dcount, nl, dl4_off);
        dl4.alloc(std::max<long long>(1, lo4[nl]));
        l4_kernel<true><<<gl, 128>>>(T, dl.p, nl, dcoll_off.p, dcoll.p, dl4_off.p, dl4.p, nullptr);
        ck(cudaGetLastError());
        const BoxLists BL{dpos.p, dcoll_off.p, dcoll.p, dl4_off.p, dl4.p};
        dt.alloc(nt);
        ck(cudaMemcpy(dt.p, tboxes.data(), nt * sizeof(int), cudaMemcpyHostToDevice));
        DBuf<int> dstatus;
        dstatus.alloc(1);
        ck(cudaMemset(dstatus.p, 0, sizeof(int)));
        const int gw = (nt + kNearWarps - 1) / kNearWarps;
        near_count_kernel<<<gw, kNearWarps * 32>>>(T, BL, dt.p, nt, dcount.p, dstatus.p);
        ck(cudaGetLastError());
        hoff = csr(dcount, nt, doff);
        raw.alloc(std::max<long long>(1, hoff[nt]));
        DBuf<int2> sorted;
        sorted.alloc(std::max<long long>(1, hoff[nt]));
        near_fill_kernel<<<gw, kNearWarps * 32>>>(T, BL, dt.p, nt, doff.p, raw.p, sorted.p, dcount.p, dstatus.p);
        ck(cudaGetLastError());
        to_host(hmerged, dcount.p, nt);
        // the merged ranges, contiguous in target-box order
        std::vector<long long> hmoff(nt + 1, 0);
        for (int i = 0; i < nt; ++i) hmoff[i + 1] = hmoff[i] + hmerged[i];
        DBuf<long long> dmoff;
        dmoff.alloc(nt + 1);
        ck(cudaMemcpy(dmoff.p, hmoff.data(), (nt + 1) * sizeof(long long), cudaMemcpyHostToDevice));
        near_b.alloc(std::max<long long>(1, hmoff[nt]));
        near_e.alloc(std::max<long long>(1, hmoff[nt]));
        compact_near_kernel<<<grid_for((int64_t)nt * 32, n_sm), 256>>>(raw.p, doff.p, dcount.p, dmoff.p, nt,
                                                                       near_b.p, near_e.p);
        ck(cudaGetLastError());
        n_near = hmoff[nt];
        int hstatus = 0;
        ck(cudaMemcpy(&hstatus, dstatus.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (hstatus) throw std::invalid_argument("near-field walk exceeded its stack");
    }
    lap(O.stats.lists_ms);

    // results to the host
    O.n_boxes = nb;
    to_host(O.level, level.p, nb);
    to_host(O.parent, parent.p, nb);
    to_host(O.src_begin, sbeg.p, nb);
    to_host(O.src_end, send.p, nb);
    std::vector<char> lf;
    to_host(lf, leaf.p, nb);
    O.is_leaf.assign(lf.begin(), lf.end());
    std::vector<double> x, y, z;
    to_host(x, cx.p, nb); to_host(y, cy.p, nb); to_host(z, cz.p, nb);
    O.center.resize(3 * (size_t)nb);
    for (int b = 0; b < nb; ++b) { O.center[b] = x[b]; O.center[nb + b] = y[b]; O.center[2 * (size_t)nb + b] = z[b]; }
    to_host(O.halfwidth, hw.p, nb);
    to_host(O.src_perm, perm, ns);
    to_host(O.ctr_box, cbox.p, nc);
    to_host(O.near_begin, near_b.p, (size_t)n_near);
    to_host(O.near_end, near_e.p, (size_t)n_near);
    O.near_start.assign(nb + 1, 0);
    for (int i = 0; i < nt; ++i) O.near_start[tboxes[i] + 1] = hmerged[i];
    for (int b = 0; b < nb; ++b) O.near_start[b + 1] += O.near_start[b];
    // target boxes are in box order, so their blocks follow near_start
    int64_t pairs = 0;
    for (int i = 0; i < nt; ++i) {
        int64_t len = 0;
        const int b = tboxes[i];
        for (int64_t k = O.near_start[b]; k < O.near_start[b + 1]; ++k) len += O.near_end[k] - O.near_begin[k];
        pairs += len * O.n_owned_ctr[b];
    }
    tsqbx_octree_stats &st = O.stats;
    st.n_boxes = nb;
    st.n_leaves = std::count(O.is_leaf.begin(), O.is_leaf.end(), 1);
    st.max_level = n_levels - 1;
    st.n_target_boxes = nt;
    st.near_nnz = (int64_t)O.near_begin.size();
    st.center_source_pairs = pairs;
    lap(st.download_ms);
}

}  // namespace

extern "C" {

int tsqbx_octree_build(int64_t n_src, const double *src_xyz, int64_t n_ctr, const double *ctr_xyz,
                       const double *ctr_radius, int n_max, double t_f, int n_mpole, int device, tsqbx_octree *out)
{
    if (!out) return TSQBX_E_INVAL;
    *out = nullptr;
    if (n_src < 0 || n_ctr < 0 || n_src > INT32_MAX - 1 || n_ctr > INT32_MAX - 1 || n_max < 1 || !(t_f >= 0.0) ||
        !std::isfinite(t_f) || n_mpole < 0 || (n_src && !src_xyz) || (n_ctr && (!ctr_xyz || !ctr_radius)))
        return TSQBX_E_INVAL;
    if (!finite_all(src_xyz, 3 * n_src) || !finite_all(ctr_xyz, 3 * n_ctr) || !finite_all(ctr_radius, n_ctr))
        return TSQBX_E_INVAL;
    for (int64_t i = 0; i < n_ctr; ++i)
        if (ctr_radius[i] < 0) return TSQBX_E_INVAL;
    tsqbx_octree_s *O = nullptr;
    try {
        DeviceGuard dg(device);
        int n_sm = 152;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) n_sm = 152;
        cudaGetLastError();
        O = new tsqbx_octree_s;
        O->n_src = n_src;
        O->n_ctr = n_ctr;
        const auto t0 = std::chrono::steady_clock::now();
        build(*O, n_src, src_xyz, n_ctr, ctr_xyz, ctr_radius, n_max, t_f, n_mpole, n_sm);
        O->stats.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = O;
        return TSQBX_OK;
    } catch (const CudaFail &f) {
        cudaGetLastError();
        delete O;
        return status_of(f.err);
    } catch (const std::bad_alloc &) {
        delete O;
        return TSQBX_E_NOMEM;
    } catch (const std::invalid_argument &) {
        delete O;
        return TSQBX_E_TOO_LARGE;
    } catch (...) {
        delete O;
        return TSQBX_E_CUDA;
    }
}

void tsqbx_octree_destroy(tsqbx_octree O) { delete O; }

int tsqbx_octree_info(tsqbx_octree O, tsqbx_octree_stats *st)
{
    if (!O || !st) return TSQBX_E_INVAL;
    *st = O->stats;
    return TSQBX_OK;
}

int tsqbx_octree_boxes(tsqbx_octree O, int32_t *level, double *center, double *halfwidth, int32_t *parent,
                       int32_t *src_begin, int32_t *src_end, int32_t *n_owned_ctr, int32_t *is_leaf)
{
    if (!O) return TSQBX_E_INVAL;
    const size_t nb = (size_t)O->n_boxes;
    auto put = [&](auto *dst, const auto &v) { if (dst && nb) std::memcpy(dst, v.data(), v.size() * sizeof(v[0])); };
    put(level, O->level);
    put(center, O->center);
    put(halfwidth, O->halfwidth);
    put(parent, O->parent);
    put(src_begin, O->src_begin);
    put(src_end, O->src_end);
    put(n_owned_ctr, O->n_owned_ctr);
    put(is_leaf, O->is_leaf);
    return TSQBX_OK;
}

int tsqbx_octree_order(tsqbx_octree O, int32_t *src_perm, int32_t *ctr_box)
{
    if (!O) return TSQBX_E_INVAL;
    if (src_perm && O->n_src) std::memcpy(src_perm, O->src_perm.data(), O->n_src * sizeof(int32_t));
    if (ctr_box && O->n_ctr) std::memcpy(ctr_box, O->ctr_box.data(), O->n_ctr * sizeof(int32_t));
    return TSQBX_OK;
}

int tsqbx_octree_near(tsqbx_octree O, int64_t *near_start, int32_t *near_begin, int32_t *near_end)
{
    if (!O) return TSQBX_E_INVAL;
    if (near_start) std::memcpy(near_start, O->near_start.data(), O->near_start.size() * sizeof(int64_t));
    const size_t n = O->near_begin.size();
    if (near_begin && n) std::memcpy(near_begin, O->near_begin.data(), n * sizeof(int32_t));
    if (near_end && n) std::memcpy(near_end, O->near_end.data(), n * sizeof(int32_t));
    return TSQBX_OK;
}

}  // extern "C"
