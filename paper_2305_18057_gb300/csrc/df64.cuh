// df64.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant
// bits (FP64 has 53) over the FP32 exponent range.  GB300 executes FP32 on
// 128 lanes per SM and clock against 2 for FP64, so FP64-class arithmetic
// built from FP32 operations can outrun the FP64 pipe.
//
// The operations are the classical error-free transformations: Knuth's
// two-sum (the exact rounding error of a + b), Dekker's fast two-sum (for
// |a| >= |b|), the two-product through a fused multiply-add (the exact error
// of a * b), and Newton's iteration for the reciprocal and the reciprocal
// square root from the single-precision approximations.  A multiply-add
// and a sum of products are formed with a single renormalisation.  Host and
// device share the code (the host forms the launch constants).
#pragma once

#include <math.h>

namespace sensei {

// keep the standard overloads visible next to the double-float ones below
using ::copysign;
using ::fabs;
using ::fma;

struct df64 {
    float hi, lo;
    df64() = default;
    // exact small constants (0.5, 1, 2, 2.5, 4 ...) and FP32 values
    __host__ __device__ constexpr explicit df64(float h) : hi(h), lo(0.0f) {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit df64(int i) : hi((float)i), lo(0.0f) {}
};

__host__ __device__ __forceinline__ float df_fma(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return fmaf(a, b, c);
#else
    return ::fmaf(a, b, c);
#endif
}

// s + e == a + b exactly (Knuth)
__host__ __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// s + e == a + b exactly when |a| >= |b| (Dekker)
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

// The sum: the exact sum of the high parts, plus the low parts, renormalised.
// Its error is below 2^-48 of the larger operand (the rounding of the low
// parts' sum), which under cancellation is an absolute, not a relative,
// bound -- ample for a residual compared at 1e-11 of its size; the
// variant that also sums the low parts' error costs twice the additions.
__host__ __device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    fast_two_sum(s, e, s, e);
    return df64(s, e);
}

__host__ __device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__host__ __device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = a.hi * b.hi;
    float e = df_fma(a.hi, b.hi, -p);        // exact error of the product of the high parts
    e = df_fma(a.hi, b.lo, df_fma(a.lo, b.hi, e));
    float s;
    fast_two_sum(p, e, s, e);
    return df64(s, e);
}

__host__ __device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__host__ __device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__host__ __device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

// a * b + c as one operation: the exact error of the high parts' product,
// the cross terms and the sum's rounding error gathered in one correction
// term, renormalised once (a product then a sum would renormalise twice)
__host__ __device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c)
{
    const float p = a.hi * b.hi;
    float pe = df_fma(a.hi, b.hi, -p);
    pe = df_fma(a.hi, b.lo, df_fma(a.lo, b.hi, pe));
    float s, e;
    two_sum(p, c.hi, s, e);
    e += pe + c.lo;
    fast_two_sum(s, e, s, e);
    return df64(s, e);
}

// Sums of products a1 b1 + a2 b2 + ... accumulated in one unnormalised pair:
// each product's exact error and each sum's rounding error gather in the
// correction term, renormalised once at the end.
struct df64_acc {
    float s, e;
};
__host__ __device__ __forceinline__ df64_acc acc_mul(df64 a, df64 b)
{
    const float p = a.hi * b.hi;
    float pe = df_fma(a.hi, b.hi, -p);
    pe = df_fma(a.hi, b.lo, df_fma(a.lo, b.hi, pe));
    return df64_acc{p, pe};
}
__host__ __device__ __forceinline__ df64_acc acc_fma(df64 a, df64 b, df64_acc x)
{
    const float p = a.hi * b.hi;
    float pe = df_fma(a.hi, b.hi, -p);
    pe = df_fma(a.hi, b.lo, df_fma(a.lo, b.hi, pe));
    float s, e;
    two_sum(x.s, p, s, e);
    return df64_acc{s, x.e + (e + pe)};
}
__host__ __device__ __forceinline__ df64 acc_done(df64_acc x)
{
    float s, e;
    fast_two_sum(x.s, x.e, s, e);
    return df64(s, e);
}

// Newton refinement of the single-precision reciprocal: r' = r + r (1 - a r)
__host__ __device__ __forceinline__ df64 rcp_df(df64 a)
{
#ifdef __CUDA_ARCH__
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(a.hi));
#else
    const float r0 = 1.0f / a.hi;
#endif
    const df64 r(r0);
    const df64 e = fma(-a, r, df64(1.0f));
    return fma(r, e, r);
}

// Newton refinement of the single-precision reciprocal square root:
// y' = y + (y / 2) (1 - a y^2)
__host__ __device__ __forceinline__ df64 rsqrt_df(df64 a)
{
#ifdef __CUDA_ARCH__
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(a.hi));
#else
    const float y0 = 1.0f / sqrtf(a.hi);
#endif
    const df64 y(y0);
    const df64 e = fma(-a, y * y, df64(1.0f));
    return fma(df64(0.5f * y0), e, y);
}

__host__ __device__ __forceinline__ df64 operator/(df64 a, df64 b) { return a * rcp_df(b); }

__host__ __device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.0f ? -a : a; }

// |a| with the sign of b (the sign of a double-float is that of its high part)
__host__ __device__ __forceinline__ df64 copysign(df64 a, df64 b)
{
    return (a.hi < 0.0f) != (b.hi < 0.0f) ? -a : a;
}

__host__ __device__ __forceinline__ double to_double(df64 a) { return (double)a.hi + (double)a.lo; }

}  // namespace sensei
