// peaks.cu -- tsqbx_measure_pipe_peaks: register-only throughput of the FP64
// and FP32 pipes, the denominators of the expansion kernels' rooflines.
//
// Each thread runs CHAINS independent fused multiply-add chains on values
// held in registers, with no memory traffic inside the loop.  Nine shapes
// (4, 8 or 16 chains per thread; 2, 4 or 8 blocks of 256 threads per SM) are
// each timed briefly; the fastest is calibrated so that one launch takes about
// kTargetMs, and the best of kRepeats timed launches (CUDA events on a stream
// of its own) is reported, counting an FMA as two flops.  The chains' results
// feed a guarded store to a __device__ sink so that the compiler keeps the
// arithmetic; the guard never holds for the seeds used.  Nothing here changes
// a setting of the GPU.
#include <algorithm>
#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "tsqbx.h"

namespace {

constexpr int kThreads = 256;
constexpr float kSearchMs = 30.f;     // per configuration while searching
constexpr float kTargetMs = 150.f;    // the final timed launches
constexpr int kRepeats = 3;

__device__ double g_sink64;
__device__ float g_sink32;

template <int CHAINS>
__global__ void __launch_bounds__(kThreads) dfma_probe(int iters, double m, double c)
{
    double a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = 1.0 + 1e-3 * i + 1e-9 * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    if (s == -1.0) g_sink64 = s;
}

template <int CHAINS>
__global__ void __launch_bounds__(kThreads) ffma_probe(int iters, float m, float c)
{
    float a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = 1.f + 1e-3f * i + 1e-7f * threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = fmaf(a[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    if (s == -1.f) g_sink32 = s;
}

// The same with packed fma.rn.f32x2: each instruction is two FP32 FMAs.
template <int CHAINS>
__global__ void __launch_bounds__(kThreads) ffma2_probe(int iters, float m, float c)
{
    using namespace tsqbx;
    f2 a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = f2_make(1.f + 1e-3f * i, 1.f - 1e-3f * i + 1e-7f * threadIdx.x);
    const f2 m2 = f2_splat(m), c2 = f2_splat(c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CHAINS; ++i) a[i] = fma2(a[i], m2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
        float x, y;
        f2_split(a[i], x, y);
        s += x + y;
    }
    if (s == -1.f) g_sink32 = s;
}

// Times `launch(iters)`: calibrates iters so that one launch takes about
// target_ms, then returns the best of `repeats` launches in *ms and the
// iteration count in *iters_out.
template <class Launch>
cudaError_t time_probe(Launch launch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float target_ms,
                       int repeats, float *ms, int *iters_out)
{
    int iters = 256;
    float t = 0.f;
    for (int cal = 0; cal < 10; ++cal) {          // grow until one launch is measurable
        cudaEventRecord(e0, s);
        launch(iters);
        cudaEventRecord(e1, s);
        cudaError_t err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) return err;
        cudaEventElapsedTime(&t, e0, e1);
        if (t >= 2.f) break;
        iters = iters * 8 > (1 << 28) ? (1 << 28) : iters * 8;
    }
    if (t > 0.f) iters = (int)std::min<double>(std::max<double>(iters * (target_ms / t), 1.0), double(1 << 30));
    float best = 0.f;
    for (int r = 0; r < repeats; ++r) {
        cudaEventRecord(e0, s);
        launch(iters);
        cudaEventRecord(e1, s);
        cudaError_t err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) return err;
        cudaEventElapsedTime(&t, e0, e1);
        if (r == 0 || t < best) best = t;
    }
    *ms = best;
    *iters_out = iters;
    return cudaGetLastError();
}

template <int C>
void launch_kind(int kind, int blocks, int n, cudaStream_t s)
{
    if (kind == 0) dfma_probe<C><<<blocks, kThreads, 0, s>>>(n, 0.9999999, 1e-8);
    else if (kind == 1) ffma_probe<C><<<blocks, kThreads, 0, s>>>(n, 0.9999f, 1e-4f);
    else ffma2_probe<C><<<blocks, kThreads, 0, s>>>(n, 0.9999f, 1e-4f);
}

void launch_shape(int kind, int chains, int blocks, int n, cudaStream_t s)
{
    if (chains == 4) launch_kind<4>(kind, blocks, n, s);
    else if (chains == 8) launch_kind<8>(kind, blocks, n, s);
    else launch_kind<16>(kind, blocks, n, s);
}

// One launch shape of one pipe (kind 0 DFMA, 1 FFMA, 2 packed FFMA), timed at
// target_ms: TFLOP/s (two flops per FMA, four per packed instruction).
cudaError_t run_shape(int kind, int chains, int blocks, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                      float target_ms, int repeats, double *tflops, float *ms_out)
{
    float ms = 0.f;
    int iters = 0;
    cudaError_t err = time_probe([&](int n) { launch_shape(kind, chains, blocks, n, s); }, s, e0, e1, target_ms,
                                 repeats, &ms, &iters);
    if (err != cudaSuccess) return err;
    const double flops_per_step = kind == 2 ? 4.0 : 2.0;
    *tflops = flops_per_step * chains * double(blocks) * kThreads * iters / (ms * 1e-3) / 1e12;
    *ms_out = ms;
    return cudaSuccess;
}

// One pipe: the nine launch shapes (4, 8 or 16 chains; 2, 4 or 8 blocks per
// SM) timed briefly, then the fastest timed again at kTargetMs.
cudaError_t probe_pipe(int kind, int sms, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double *tflops,
                       float *ms_out)
{
    const int chains[3] = {4, 8, 16}, per_sm[3] = {2, 4, 8};
    double best = 0.0;
    int best_c = 8, best_b = 4;
    for (int c : chains)
        for (int b : per_sm) {
            double tf = 0.0;
            float ms = 0.f;
            cudaError_t err = run_shape(kind, c, sms * b, s, e0, e1, kSearchMs, 2, &tf, &ms);
            if (err != cudaSuccess) return err;
            if (tf > best) { best = tf; best_c = c; best_b = b; }
        }
    return run_shape(kind, best_c, sms * best_b, s, e0, e1, kTargetMs, kRepeats, tflops, ms_out);
}

}  // namespace

extern "C" int tsqbx_measure_pipe_peaks(int device, tsqbx_pipe_peaks *out)
{
    if (!out) return TSQBX_E_INVAL;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess) { cudaGetLastError(); return TSQBX_E_CUDA; }
    if (device < 0 || device >= n_dev) return TSQBX_E_INVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return TSQBX_E_CUDA; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    double tf64 = 0.0, tf32 = 0.0, tf32x2 = 0.0;
    float ms64 = 0.f, ms32 = 0.f, ms32x2 = 0.f;
    if (err == cudaSuccess) err = probe_pipe(0, sms, s, e0, e1, &tf64, &ms64);
    if (err == cudaSuccess) err = probe_pipe(1, sms, s, e0, e1, &tf32, &ms32);
    if (err == cudaSuccess) err = probe_pipe(2, sms, s, e0, e1, &tf32x2, &ms32x2);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaSetDevice(prev);
    if (err != cudaSuccess) { cudaGetLastError(); return TSQBX_E_CUDA; }
    out->sm_count = sms;
    out->fp64_tflops = tf64;
    out->fp32_tflops = tf32;
    out->fp32x2_tflops = tf32x2;
    out->ms_fp64 = ms64;
    out->ms_fp32 = ms32;
    out->ms_fp32x2 = ms32x2;
    return TSQBX_OK;
}
