// sgpe_df.cuh -- "double-float" arithmetic: a real number held as the
// unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2), about 48
// significant bits, computed entirely on the FP32 pipe.
//
// Why: GB300 executes FP64 at about 1/60 of its FP32 rate (a warp's FP64
// instruction occupies its SM sub-partition for ~64-80 cycles), so the
// complex128 step is bound by the FP64 pipe. A double-float operation costs
// 3-15 FP32 instructions, each one cycle per warp, which is several times
// cheaper than one FP64 instruction while keeping the step's error near
// 1e-13, far inside the 1e-10 FP64 parity bar.
//
// Building blocks (error-free transformations with FMA, after Dekker and
// Knuth): two_sum gives s + e = a + b exactly; fast_two_sum the same when
// |a| >= |b|; two_prod gives p + e = a * b exactly (e from one FMA).
// Addition is the "sloppy" variant (error relative to |a| + |b|, adequate
// here: no result of the step depends on a cancellation of large terms),
// multiplication adds the two cross terms before renormalising.
// The exponent range is FP32's; values below ~1e-38 flush towards zero and
// lose their low part, which is far below anything the step resolves.
#pragma once
#include <cuda_runtime.h>

namespace sgpe {

// The double-float fma below must not hide the built-in overloads inside this namespace.
using ::fma;
using ::fmaf;

struct df {
    float hi, lo;
    __host__ __device__ df() {}
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit constexpr df(int v) : hi((float)v), lo(0.0f) {}
};

// Split a double into hi + lo (host or device; on the device it costs FP64
// instructions, so kernels take precomputed pairs or compile-time constants).
__host__ __device__ constexpr df df_from(double d) { return df((float)d, (float)(d - (double)(float)d)); }
__host__ __device__ inline double df_to(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float t = s - a;
    return df(s, (a - (s - t)) + (b - t));
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = a + b;
    return df(s, b - (s - a));
}
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = a * b;
    return df(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator+(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    float e = fmaf(a.hi, b.lo, p.lo);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p.hi, e);
}
// a * b + c with one renormalisation of the product's cross terms folded into the sum
__device__ __forceinline__ df fma(df a, df b, df c) {
    df p = two_prod(a.hi, b.hi);
    float e = fmaf(a.hi, b.lo, p.lo);
    e = fmaf(a.lo, b.hi, e);
    df s = two_sum(p.hi, c.hi);
    return fast_two_sum(s.hi, s.lo + (e + c.lo));
}

// 1/sqrt(a) for a > 0: FP32 estimate, then two Newton steps y <- y (3 - a y^2)/2
// in double-float (error ~2^-23, then ~2^-45, then the format's ~2^-48).
__device__ __forceinline__ df df_rsqrt(df a) {
    df y = df(rsqrtf(a.hi), 0.0f);
#pragma unroll
    for (int it = 0; it < 2; it++) {
        const df ay2 = (a * y) * y;
        const df h = df(1.5f, 0.0f) - df(0.5f * ay2.hi, 0.5f * ay2.lo);
        y = y * h;
    }
    return y;
}

// a + b for an FP32 b (one error-free sum fewer than a full double-float add).
__device__ __forceinline__ df add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

// exp(x) for |x| < 2^-6: 1 + x(1 + x(1/2 + x(1/6 + r))) with the tail
// r = x/24 + x^2/120 + x^3/720 in FP32 (|r| < 2^-11; its FP32 rounding, scaled
// by x^3 < 2^-18, stays below 2^-60) and the outer Horner steps in
// double-float; truncation (x^7/7! < 2^-54) below the format's 2^-48. Other
// arguments through FP64.
__device__ __forceinline__ df exp_small(df x) {
    if (fabsf(x.hi) < 0.015625f) {
        const float xf = x.hi;
        const float r = xf * fmaf(xf, fmaf(xf, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f);
        constexpr df c6 = df_from(1.0 / 6.0);
        df p = add_f(c6, r);
        p = fma(p, x, df(0.5f, 0.0f));
        p = fma(p, x, df(1.0f, 0.0f));
        return fma(p, x, df(1.0f, 0.0f));
    }
    return df_from(exp(df_to(x)));
}

// (sin x, cos x) for |x| < 2^-6, t = x^2 < 2^-12: sin(x)/x = 1 - t(1/6 - rs),
// cos(x) = 1 - t(1/2 - t(1/24 - rc)), with the tails rs = t/120 - t^2/5040 and
// rc = t/720 in FP32 (their rounding, scaled by t or t^2, below 2^-60); the
// outer steps in double-float. Other arguments through FP64.
__device__ __forceinline__ void sincos_small(df x, df* s, df* c) {
    if (fabsf(x.hi) < 0.015625f) {
        const df mt = -(x * x);
        const float tf = x.hi * x.hi;
        const float rs = tf * fmaf(-tf, 1.0f / 5040.0f, 1.0f / 120.0f);
        const float rc = tf * (1.0f / 720.0f);
        constexpr df c6 = df_from(1.0 / 6.0), c24 = df_from(1.0 / 24.0);
        df ps = add_f(c6, -rs);                  // 1/6 - t/120 + t^2/5040
        ps = fma(ps, mt, df(1.0f, 0.0f));        // sin(x)/x
        df pc = add_f(c24, -rc);                 // 1/24 - t/720
        pc = fma(pc, mt, df(0.5f, 0.0f));        // 1/2 - t/24 + t^2/720
        pc = fma(pc, mt, df(1.0f, 0.0f));        // cos(x)
        *s = ps * x;
        *c = pc;
        return;
    }
    double sd, cd;
    sincos(df_to(x), &sd, &cd);
    *s = df_from(sd);
    *c = df_from(cd);
}

}  // namespace sgpe
