// Double-float arithmetic: a value carried as an unevaluated sum hi + lo of
// two FP32 numbers, |lo| <= ~ulp(hi), for ~48 bits of significand on the FP32
// pipe (GB300's FP64 pipe runs at 1/64 of the FP32 rate).  The error-free
// transformations are the published ones: Knuth's two-sum, Dekker's fast
// two-sum (|a| >= |b|), and the FMA form of Dekker's two-product; the
// products below leave their pairs unnormalised (the next operation takes hi
// and lo as they are), which costs at most a few units of 2^-48 in relative
// error over a chain of products.  Every operation rounds to nearest and
// takes no fused contraction of its own (the __f*_rn intrinsics).
#pragma once

#include <cuda_runtime.h>

namespace lisa {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

// a + b exactly, as (s, e) (Knuth).
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// a + b exactly for |a| >= |b| (Dekker).
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

// a * b exactly, as (p, e).
__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return df{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_renorm(df a) { return fast_two_sum(a.hi, a.lo); }

__device__ __forceinline__ df df_add(df a, df b)
{
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df{-b.hi, -b.lo}); }

// Product, left unnormalised: (a.hi b.hi rounded, its exact error plus the
// cross terms).
__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df{p, e};
}

__device__ __forceinline__ df df_mul_f(df a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    return df{p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p))};
}

// a * b + c (c a double-float), normalised.
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_renorm(df_mul(a, b)), c); }

__device__ __forceinline__ df df_from_double(double d)
{
    const float hi = __double2float_rn(d);
    return df{hi, __double2float_rn(d - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// Horner evaluation of sum_{k=0..N-1} c_k u^k with double-float coefficients
// (c[k] = (hi, lo)) at an FP32 argument u.
template <int N>
__device__ __forceinline__ df df_horner(const df* c, float u)
{
    df r = c[N - 1];
#pragma unroll
    for (int k = N - 2; k >= 0; --k) r = df_add(df_renorm(df_mul_f(r, u)), c[k]);
    return r;
}

// The same sum with only c_0 .. c_{K-1} in double-float: the tail
// sum_{k>=K} c_k u^k is formed from the coefficients' high parts in FP32, for
// series whose tail is small enough that its FP32 rounding is below the
// accuracy the caller needs.
template <int N, int K>
__device__ __forceinline__ df df_horner_tail(const df* c, float u)
{
    float r = c[N - 1].hi;
#pragma unroll
    for (int k = N - 2; k >= K; --k) r = __fmaf_rn(r, u, c[k].hi);
    df acc = df_add(c[K - 1], df{__fmul_rn(r, u), 0.f});
#pragma unroll
    for (int k = K - 2; k >= 0; --k) acc = df_add(df_renorm(df_mul_f(acc, u)), c[k]);
    return acc;
}

}  // namespace lisa
