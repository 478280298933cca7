// noalloc.cu -- tsqbx_eval_noalloc: a Laplace FP64 evaluation that allocates
// nothing, for callers that cannot call cudaMalloc.
//
// Who needs it: code that hands this library memory it already owns and must
// not allocate more -- e.g. a host program whose device memory is entirely
// managed by its own pool or arena (a second allocator would fight it or fail),
// or a latency-critical loop that cannot accept cudaMalloc's implicit device
// synchronisation.  Such a caller cannot build a plan (plan creation allocates
// device buffers), so this entry point takes the geometry, the pair lists, the
// density and the outputs directly as device arrays.
//
// Its only scratch -- w_s mu_s for every source and a status word -- lives in
// one file-scope __device__ array of fixed size (kScratchDoubles doubles,
// 8 MiB), reserved on every GPU that loads the library until the process
// exits.  Every call shares that array: calls that overlap on the GPU (on
// different streams, or from several host threads) race on it and must be
// serialised by the caller.  The array keeps the last call's contents; the
// status word is cleared at the start of every call, and the w mu part is
// fully rewritten for the call's sources before it is read.
#include <mutex>
#include <utility>

#include "internal.cuh"
#include "tsqbx.h"

namespace {

using namespace tsqbx;

// 32 leading doubles (256 bytes) hold the status word; the rest holds w mu.
constexpr int64_t kScratchDoubles = int64_t(1) << 20;
constexpr int64_t kStatusDoubles = 32;
static_assert(TSQBX_NOALLOC_MAX_SRC == kScratchDoubles - kStatusDoubles,
              "header limit must match the scratch array");

static __device__ __align__(256) double noalloc_scratch[kScratchDoubles];

struct RawGeom {
    int64_t n_src, n_ctr, n_tgt, n_group;
    const double *src_xyz, *src_weight, *src_normal;
    const double *ctr_xyz, *tgt_xyz;
    const int32_t *tgt_center, *ctr_group;
    const int64_t *group_range_start;
    const int32_t *range_begin, *range_end;
};

__global__ void noalloc_prep(const double *w, const double *mu, int64_t n, double *wmu)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        wmu[i] = w[i] * mu[i];
}

// One warp per target; lanes stride through the sources of each listed range
// (coalesced structure-of-arrays loads) and run the scaled Legendre recurrence
// forward (Q_n = kappa_n T_n, eq. tsqbx), with the double layer from the
// derivative recurrence and its closing sums (Appendix A); a butterfly shuffle
// combines the lanes.  Status bits: 1 = an index out of range (the access is
// skipped), 2 = a source on its center (R = 0, where the expansion does not
// exist; the pair is skipped).  Divergent pairs (|t-c| >= |s-c|) are not
// looked for: such a pair is summed like any other.
template <int P, bool DLP>
__global__ void __launch_bounds__(128)
noalloc_laplace_fp64(const RawGeom g, const double *wmu, unsigned long long *status,
                     double *out_slp, double *out_dlp)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= g.n_tgt) return;                              // warp-uniform
    double acc_s = 0.0, acc_d = 0.0;
    const int32_t c = g.tgt_center[t];
    bool ok = c >= 0 && c < g.n_ctr;
    const int32_t q = ok ? g.ctr_group[c] : 0;
    ok = ok && q >= 0 && q < g.n_group;
    int64_t r0 = 0, r1 = 0;
    if (ok) {
        r0 = g.group_range_start[q];
        r1 = g.group_range_start[q + 1];
        ok = r0 >= 0 && r1 >= r0 && r1 <= g.group_range_start[g.n_group];
    }
    if (!ok) {
        if (lane == 0) atomicOr(status, 1ull);
        r1 = r0;
    }
    double cx = 0, cy = 0, cz = 0, ex = 0, ey = 0, ez = 0;
    if (ok) {
        cx = g.ctr_xyz[c]; cy = g.ctr_xyz[g.n_ctr + c]; cz = g.ctr_xyz[2 * g.n_ctr + c];
        ex = g.tgt_xyz[t] - cx; ey = g.tgt_xyz[g.n_tgt + t] - cy; ez = g.tgt_xyz[2 * g.n_tgt + t] - cz;
    }
    const double rho2 = fma(ex, ex, fma(ey, ey, ez * ez));
    for (int64_t r = r0; r < r1; ++r) {
        int32_t b = g.range_begin[r], e = g.range_end[r];
        if (b < 0 || e < b || e > g.n_src) {
            if (lane == 0) atomicOr(status, 1ull);
            continue;
        }
        for (int32_t s = b + lane; s < e; s += 32) {
            const double dx = g.src_xyz[s] - cx, dy = g.src_xyz[g.n_src + s] - cy,
                         dz = g.src_xyz[2 * g.n_src + s] - cz;
            const double wm = wmu[s];
            const double R2 = fma(dx, dx, fma(dy, dy, dz * dz));
            if (!(R2 > 0.0)) {              // source on the center: the expansion does not exist
                atomicOr(status, 2ull);
                continue;
            }
            const double rinv = rsqrt(R2);
            const double r2inv = rinv * rinv;
            const double qx = fma(dx, ex, fma(dy, ey, dz * ez)) * r2inv;
            const double q2 = rho2 * r2inv;
            double S0 = 1.0, S2 = 0.0;
            double Tm = 1.0, Tc = 1.0, Dm = 0.0, Dc = 0.0;
            if (P >= 1) { S0 += qx; S2 = 1.0; Tc = qx; Dc = 1.0; }
#pragma unroll
            for (int n = 1; n < P; ++n) {
                const double Tn = fma(qx, Tc, -(rec_beta(n) * q2) * Tm);
                S0 = fma(rec_kappa(n + 1), Tn, S0);
                if (DLP) {
                    const double Dn = fma(q2, Dm, ((2.0 * n + 1.0) * rec_kappa(n)) * Tc);
                    S2 += Dn;
                    Dm = Dc; Dc = Dn;
                }
                Tm = Tc; Tc = Tn;
            }
            acc_s = fma(wm * rinv, S0, acc_s);
            if (DLP) {
                const double nx = g.src_normal[s], ny = g.src_normal[g.n_src + s],
                             nz = g.src_normal[2 * g.n_src + s];
                const double Dp1 = fma(q2, Dm, ((2.0 * P + 1.0) * rec_kappa(P)) * Tc);
                const double S1 = 0.5 * (fma(-q2, S2, S2) + Dp1 + fma(q2, Dc, S0));
                const double a = fma(dx, nx, fma(dy, ny, dz * nz));
                const double bb = fma(ex, nx, fma(ey, ny, ez * nz));
                acc_d = fma(wm * rinv * r2inv, fma(-a, S1, fma(-a, qx, bb) * S2), acc_d);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc_s += __shfl_xor_sync(0xffffffffu, acc_s, off);
        acc_d += __shfl_xor_sync(0xffffffffu, acc_d, off);
    }
    if (lane == 0) {
        if (out_slp) out_slp[t] = acc_s * kInv4Pi;
        if (DLP && out_dlp) out_dlp[t] = acc_d * kInv4Pi;
    }
}

template <int P>
void launch(bool dlp, const RawGeom &g, const double *wmu, unsigned long long *st, double *os,
            double *od, cudaStream_t s)
{
    const int64_t blocks = (g.n_tgt * 32 + 127) / 128;
    if (blocks == 0) return;
    if (dlp) noalloc_laplace_fp64<P, true><<<(unsigned)blocks, 128, 0, s>>>(g, wmu, st, os, od);
    else     noalloc_laplace_fp64<P, false><<<(unsigned)blocks, 128, 0, s>>>(g, wmu, st, os, od);
}

template <int... Ps>
void dispatch(int p, bool dlp, const RawGeom &g, const double *wmu, unsigned long long *st,
              double *os, double *od, cudaStream_t s, std::integer_sequence<int, Ps...>)
{
    ((p == Ps ? (launch<Ps>(dlp, g, wmu, st, os, od, s), 0) : 0), ...);
}

// Device address of noalloc_scratch, looked up once per device (with that
// device current) by the first call on it.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int tsqbx_eval_noalloc(const tsqbx_geometry *d_geometry, int p, uint32_t layers,
                                  const double *d_density, double *d_out_slp, double *d_out_dlp,
                                  void *stream)
{
    const tsqbx_geometry *G = d_geometry;
    if (!G || p < 0 || p > TSQBX_P_MAX || layers == 0 ||
        (layers & ~(uint32_t)(TSQBX_SLP | TSQBX_DLP)))
        return TSQBX_E_INVAL;
    if (G->n_src < 0 || G->n_ctr < 0 || G->n_tgt < 0 || G->n_group < 0 || G->n_tgt > INT32_MAX)
        return TSQBX_E_INVAL;
    if (G->n_src > TSQBX_NOALLOC_MAX_SRC) return TSQBX_E_TOO_LARGE;
    const bool dlp = (layers & TSQBX_DLP) != 0;
    if ((G->n_src && (!G->src_xyz || !G->src_weight || !d_density)) ||
        (dlp && G->n_src && !G->src_normal) || (G->n_ctr && (!G->ctr_xyz || !G->ctr_group)) ||
        (G->n_tgt && (!G->tgt_xyz || !G->tgt_center)) || !G->group_range_start ||
        (G->n_group && (!G->range_begin || !G->range_end)) ||
        ((layers & TSQBX_SLP) && G->n_tgt && !d_out_slp) || (dlp && G->n_tgt && !d_out_dlp))
        return TSQBX_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return TSQBX_E_CUDA; }
    double *scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) { cudaGetLastError(); return TSQBX_E_CUDA; }
    unsigned long long *status = reinterpret_cast<unsigned long long *>(scratch);
    double *wmu = scratch + kStatusDoubles;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    RawGeom g{G->n_src, G->n_ctr, G->n_tgt, G->n_group, G->src_xyz, G->src_weight, G->src_normal,
              G->ctr_xyz, G->tgt_xyz, G->tgt_center, G->ctr_group, G->group_range_start,
              G->range_begin, G->range_end};
    if (cudaMemsetAsync(status, 0, sizeof(unsigned long long), s) != cudaSuccess) {
        cudaGetLastError();
        return TSQBX_E_CUDA;
    }
    if (G->n_src > 0) {
        const int blocks = (int)std::min<int64_t>((G->n_src + 255) / 256, 152 * 16);
        noalloc_prep<<<blocks, 256, 0, s>>>(G->src_weight, d_density, G->n_src, wmu);
    }
    dispatch(p, dlp, g, wmu, status, (layers & TSQBX_SLP) ? d_out_slp : nullptr,
             dlp ? d_out_dlp : nullptr, s, std::make_integer_sequence<int, TSQBX_P_MAX + 1>{});
    unsigned long long h_status = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h_status, status, sizeof(h_status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cudaGetLastError(); return TSQBX_E_CUDA; }
    return h_status ? TSQBX_E_KERNEL : TSQBX_OK;
}
