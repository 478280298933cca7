// f32x2.cuh -- packed pairs of FP32 values and their arithmetic through the
// sm_100-family packed instructions (add/sub/mul/fma .rn.f32x2): two
// independent round-to-nearest FP32 operations per instruction issued.  The
// FP32 pipe's flop rate is the same as for scalar operations; what halves is
// the number of issue slots, which is what limits the mixed-precision kernel.
// Every operation rounds once (explicit .rn: nothing is contracted).
#pragma once

#include <cuda_runtime.h>

namespace tsqbx {

struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 f2_make(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2 f2_splat(float a) { return f2_make(a, a); }
__device__ __forceinline__ void f2_split(f2 r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r.v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return d;
}
// 1/sqrt(x) and 1/x as single special-function-unit instructions (PTX
// rsqrt.approx.ftz.f32, rcp.approx.ftz.f32; rcp within 1 ulp).  Unlike
// rsqrtf they carry no handling of subnormal arguments, which flush to zero
// (so give +inf): the kernels take them of squared center-source distances,
// which for any surface of size 1e-3 .. 1e3 lie far above FP32's subnormal
// range (below 1.2e-38).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Both halves of a float4's (x, y) or (z, w) as one packed value.
__device__ __forceinline__ f2 f2_xy(const float4 &q) { return f2_make(q.x, q.y); }
__device__ __forceinline__ f2 f2_zw(const float4 &q) { return f2_make(q.z, q.w); }

// Kahan-compensated accumulation of two independent sums at once.
__device__ __forceinline__ void kahan_add2(f2 &s, f2 &c, f2 x)
{
    const f2 y = sub2(x, c);
    const f2 t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
}

}  // namespace tsqbx
