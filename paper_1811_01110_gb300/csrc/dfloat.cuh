// dfloat.cuh -- double-float ("df64") arithmetic: a value is the unevaluated
// sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, giving a ~48-bit
// significand computed entirely on the FP32 pipes.  On GB300 the FP32 pipes
// run ~61x the FP64 rate, so FP64-class accuracy is cheaper this way.
//
// Building blocks are the error-free transformations (Knuth's TwoSum,
// Dekker's FastTwoSum, FMA-based TwoProd) and the double-word algorithms of
// Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic" (ACM TOMS 2017):
//   df_add   -- their "sloppy" DWPlusDW: error <= 2^-46 (|x| + |y|);
//   df_mul   -- DWTimesDW (FMA variant): relative error <= 5 * 2^-48;
//   df_mul_f -- DWTimesFP: relative error <= 2 * 2^-48.
// All steps use explicit round-to-nearest intrinsics so the compiler neither
// contracts nor reassociates them.  1/sqrt is rsqrt.approx refined by two Newton
// steps y <- y + y (1 - a y^2) / 2 evaluated in double-float.
#pragma once

#include <cuda_runtime.h>

#include "f32x2.cuh"

namespace tsqbx {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y)
{
    const float ch = __fmul_rn(x.hi, y.hi);
    const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
    const float tl = __fmul_rn(x.hi, y.lo);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl);
    return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

__device__ __forceinline__ df df_mul_f(df x, float y)
{
    const float ch = __fmul_rn(x.hi, y);
    const float cl1 = __fmaf_rn(x.hi, y, -ch);
    return fast_two_sum(ch, __fmaf_rn(x.lo, y, cl1));
}

__device__ __forceinline__ df df_from_double(double v)
{
    const float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

// 1/sqrt(a), a > 0 (relative error ~2^-46)
__device__ __forceinline__ df df_rsqrt(df a)
{
    const float r0 = rsqrt_approx(a.hi);
    const df ar0 = df_mul(a, two_prod(r0, r0));
    const df h0 = df_add(df{1.f, 0.f}, df_neg(ar0));
    const df r1 = fast_two_sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), h0.hi));
    const df ar1 = df_mul(a, df_mul(r1, r1));
    const df h1 = df_add(df{1.f, 0.f}, df_neg(ar1));
    return df_add(r1, df_mul_f(r1, __fmul_rn(0.5f, h1.hi)));
}

// Compile-time split of a double constant into hi + lo floats.
struct dfc {
    float hi, lo;
};
__host__ __device__ constexpr dfc df_const(double v)
{
    return dfc{(float)v, (float)(v - (double)(float)v)};
}
__device__ __forceinline__ df df_of(dfc c) { return df{c.hi, c.lo}; }

// Product with a compile-time constant: a constant that is itself a float
// (lo = 0, e.g. the dyadic lambda_n of low order) takes the double-word-
// times-float algorithm, which skips the products by its zero lo part (IEEE
// arithmetic does not fold x * 0).  The test folds away once the constant is
// known.
__device__ __forceinline__ df df_mul_c(dfc c, df x) { return c.lo == 0.f ? df_mul_f(x, c.hi) : df_mul(df_of(c), x); }

}  // namespace tsqbx
