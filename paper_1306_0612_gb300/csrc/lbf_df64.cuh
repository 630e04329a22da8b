// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats
// (|lo| <= ulp(hi)/2), about 48 significant bits.  On this GPU the float pipes issue
// 64 times faster than the double pipe, so the accurate FMM operator runs its
// expansions, translations and near field in this type.
//
// Built on the error-free transformations of floating-point arithmetic:
//   two_sum (Knuth):        s + e = a + b exactly, s = fl(a + b)
//   fast_two_sum (Dekker):  the same when |a| >= |b|, three operations
//   two_prod (with FMA):    p + e = a * b exactly, p = fl(a * b), e = fma(a, b, -p)
// Addition is the "sloppy" variant (error O(2^-48 (|a| + |b|)), the same form as a
// double sum's bound); multiplication adds the cross terms hi*lo before renormalising.
#pragma once

#include <cuda_runtime.h>

struct __align__(8) df64 {
    float hi, lo;
    df64() = default;  // trivial: usable in __shared__ arrays
    __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ df64(float f) : hi(f), lo(0.f) {}
    __host__ __device__ df64(int i) : df64((double)i) {}
    __host__ __device__ df64(float h, float l, int) : hi(h), lo(l) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ df64 df_fast(float a, float b)  // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)), 0);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    float s, e;
    df_two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_fast(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo, 0); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast(p, e);
}

// a * b + c
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    df_two_sum(p, c.hi, s, t);
    t = __fadd_rn(t, __fadd_rn(e, c.lo));
    return df_fast(s, t);
}

__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

// 1/a: one Newton step x + x (1 - a x) from the float reciprocal (24 -> ~48 bits)
__device__ __forceinline__ df64 df_rcp(df64 a)
{
    float x = __frcp_rn(a.hi);
    df64 xd(x);
    df64 r = df_fma(-a, xd, df64(1.0f));
    return df_fma(xd, r, xd);
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return a * df_rcp(b); }

// the float nearest to hi + lo
__device__ __forceinline__ float df_round(df64 a) { return __fadd_rn(a.hi, a.lo); }

// exact scaling by a power of two
__device__ __forceinline__ df64 df_ldexp(df64 a, float p2) { return df64(a.hi * p2, a.lo * p2, 0); }

__device__ __forceinline__ df64 __shfl_xor_sync(unsigned mask, df64 v, int lane, int width = 32)
{
    return df64(__shfl_xor_sync(mask, v.hi, lane, width), __shfl_xor_sync(mask, v.lo, lane, width), 0);
}
__device__ __forceinline__ df64 __shfl_sync(unsigned mask, df64 v, int lane, int width = 32)
{
    return df64(__shfl_sync(mask, v.hi, lane, width), __shfl_sync(mask, v.lo, lane, width), 0);
}
__device__ __forceinline__ df64 __shfl_down_sync(unsigned mask, df64 v, unsigned d, int width = 32)
{
    return df64(__shfl_down_sync(mask, v.hi, d, width), __shfl_down_sync(mask, v.lo, d, width), 0);
}
