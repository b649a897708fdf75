// sgpe_device.cuh -- device arithmetic shared by the step, observable and
// adjoint kernels: complex helpers, small-argument exponential / sine-cosine
// polynomials, and the per-point substeps of the split-step scheme of
// arXiv:2009.13507 (SO: Appendix A Eqs. (p1)-(p2); CALCNU: the diagonal terms
// of Eqs. (1)-(2); HERM: Appendix A Eqs. (nu), (11)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "sgpe_df.cuh"

namespace sgpe {

// Storage element of one complex number per arithmetic type R: complex128,
// complex64, and the double-float pair (re.hi, re.lo, im.hi, im.lo).
template <typename R> struct V2;
template <> struct V2<double> { using T = double2; };
template <> struct V2<float> { using T = float2; };
template <> struct V2<df> { using T = float4; };

template <typename R> struct cx {
    R re, im;
};

__device__ __forceinline__ cx<double> unpack(double2 v) { return {v.x, v.y}; }
__device__ __forceinline__ cx<float> unpack(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ cx<df> unpack(float4 v) { return {df(v.x, v.y), df(v.z, v.w)}; }
__device__ __forceinline__ double2 pack(cx<double> a) { return make_double2(a.re, a.im); }
__device__ __forceinline__ float2 pack(cx<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ float4 pack(cx<df> a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }

// The value as a double (observables, norms: FP64 arithmetic).
__device__ __forceinline__ double dbl(double x) { return x; }
__device__ __forceinline__ double dbl(float x) { return (double)x; }
__device__ __forceinline__ double dbl(df x) { return df_to(x); }
// A double rounded to R (FP64 conversion: off the per-point path).
template <typename R> __device__ __forceinline__ R to_r(double x) { return (R)x; }
template <> __device__ __forceinline__ df to_r<df>(double x) { return df_from(x); }
template <typename R> constexpr bool is_f32() { return sizeof(R) == 4; }
// A double-float value as R (only meaningful for R = df; the others take its sum).
template <typename R> __device__ __forceinline__ R to_r_df(df x) { return (R)df_to(x); }
template <> __device__ __forceinline__ df to_r_df<df>(df x) { return x; }

template <typename R> __device__ __forceinline__ cx<R> add(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ cx<R> sub(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ cx<R> scl(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> __device__ __forceinline__ cx<R> mul(cx<R> a, cx<R> b) {
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
// conj(a) * b
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    return {fma(a.re, b.re, a.im * b.im), fma(a.re, b.im, -a.im * b.re)};
}
template <typename R> __device__ __forceinline__ R nrm(cx<R> a) { return fma(a.re, a.re, a.im * a.im); }
template <typename R> __device__ __forceinline__ cx<R> cj(cx<R> a) { return {a.re, -a.im}; }
// a + s*b (s real)
template <typename R> __device__ __forceinline__ cx<R> axpy(R s, cx<R> b, cx<R> a) {
    return {fma(s, b.re, a.re), fma(s, b.im, a.im)};
}
// a + s*b (s complex)
template <typename R> __device__ __forceinline__ cx<R> caxpy(cx<R> s, cx<R> b, cx<R> a) {
    return {fma(s.re, b.re, fma(-s.im, b.im, a.re)), fma(s.re, b.im, fma(s.im, b.re, a.im))};
}

template <typename R> __device__ __forceinline__ cx<R> ld(const typename V2<R>::T* p, size_t i) {
    return unpack(__ldg(p + i));
}
template <typename R> __device__ __forceinline__ cx<R> ldc(const typename V2<R>::T* p, size_t i) {
    return unpack(__ldcg(p + i));  // L2 only: data written earlier in this kernel's grid or stream
}
template <typename R> __device__ __forceinline__ void st(typename V2<R>::T* p, size_t i, cx<R> a) { p[i] = pack(a); }

// ---------------------------------------------------------------------------
// exp(x) and (cos x, sin x) for the phase factors.
//
// FP64: GB300 executes FP64 at about 1/60 of its FP32 rate, so the library
// exponential / sincos (range reduction plus a long polynomial) would dominate
// the pointwise substeps. Every argument here is dt times an energy, normally
// below 1/64 in magnitude, where a truncated Taylor series evaluated by
// Horner's rule is accurate to under an ulp:
//   exp(x) = sum_{n<=6} x^n/n!   (|x| <= 2^-6: first omitted term < 4.5e-17, 0.2 ulp of 1)
//   sin(x) = x sum_{n<=3} (-x^2)^n/(2n+1)!   (omitted < 1e-20)
//   cos(x) = sum_{n<=3} (-x^2)^n/(2n)!       (omitted < 9e-20)
// Larger arguments take CUDA's exp / sincos. The range test reads the high
// word of the double on the integer pipe: |x| < 2^-6 iff (hi & 0x7fffffff) < 0x3F900000.
// FP32: CUDA's expf / sincosf (full-range, FP32 pipe).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool small_arg(double x) {
    return (unsigned)(__double2hiint(x) & 0x7fffffff) < 0x3F900000u;  // |x| < 2^-6
}

__device__ __forceinline__ double exp_small(double x) {
    if (small_arg(x)) {
        double p = 1.0 / 720.0;
        p = fma(p, x, 1.0 / 120.0);
        p = fma(p, x, 1.0 / 24.0);
        p = fma(p, x, 1.0 / 6.0);
        p = fma(p, x, 0.5);
        p = fma(p, x, 1.0);
        return fma(p, x, 1.0);
    }
    return exp(x);
}
__device__ __forceinline__ float exp_small(float x) { return expf(x); }

// exp(x) - 1 in FP32 for the complex64 CALCNU factor, written out from the
// mathematics: Cody-Waite reduction x = k ln2 + r with |r| <= ln2/2 (ln2 split
// into a 12-bit head, whose product with k is exact for |k| < 2^12, and the
// rest), the Taylor series of expm1(r) through r^8/8! (the omitted terms stay
// below 6e-10 |r|, 0.01 ulp), and expm1(x) = 2^k expm1(r) + (2^k - 1) in one
// fused multiply-add (2^k - 1 is exact for |k| <= 24; k = 0 returns the series
// itself). The argument is clamped to [-87.3, 89] so that 2^k stays a normal
// number or becomes infinity (x > 88.72: the true result overflows too); the
// clamp compares, so a NaN argument stays NaN.
__device__ __forceinline__ float expm1_cw(float x) {
    x = x < -87.3f ? -87.3f : x;
    x = x > 89.0f ? 89.0f : x;
    const float kf = rintf(x * 1.44269504088896341f);  // nearest integer to x / ln2
    float r = fmaf(-kf, 0.693145751953125f, x);         // ln2 head: 2839 / 4096
    r = fmaf(-kf, 1.42860682030941723e-6f, r);          // ln2 - head
    float q = 1.0f / 40320.0f;
    q = fmaf(q, r, 1.0f / 5040.0f);
    q = fmaf(q, r, 1.0f / 720.0f);
    q = fmaf(q, r, 1.0f / 120.0f);
    q = fmaf(q, r, 1.0f / 24.0f);
    q = fmaf(q, r, 1.0f / 6.0f);
    q = fmaf(q, r, 0.5f);
    const float e = fmaf(q, r * r, r);  // expm1(r)
    const float t = __int_as_float(((int)kf + 127) << 23);  // 2^k
    return fmaf(t, e, t - 1.0f);
}

// Two FP32 numbers as one operand of the packed FP32x2 instructions (add, sub,
// mul and fma on both lanes at once, each lane rounded as the scalar
// instruction rounds it). The complex64 pointwise kernel evaluates its two grid
// points (ix, ix + 1) as one pair, so each arithmetic instruction of the
// substeps serves both points.
struct f32x2 {
    float2 v;
    f32x2() = default;
    __device__ __forceinline__ f32x2(float2 a) : v(a) {}
    __device__ __forceinline__ f32x2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit f32x2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ explicit f32x2(int a) : v(make_float2((float)a, (float)a)) {}
};
template <typename R> constexpr bool is_pair() { return std::is_same<R, f32x2>::value; }
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) { return __fadd2_rn(a.v, b.v); }
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) { return __fmul2_rn(a.v, b.v); }
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) {
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.v.x), "f"(a.v.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.v.x), "f"(b.v.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(rd));
    return f32x2(x, y);
}
// -a, an exact sign change of both lanes
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return __fmul2_rn(a.v, make_float2(-1.0f, -1.0f)); }
__device__ __forceinline__ f32x2 fma(f32x2 a, f32x2 b, f32x2 c) { return __ffma2_rn(a.v, b.v, c.v); }

// expm1_cw on both lanes: the clamps, the rounding to the nearest integer and the
// exponent of 2^k per lane, the rest on the packed instructions (each lane the
// same operations in the same order as expm1_cw).
__device__ __forceinline__ f32x2 expm1_cw(f32x2 x) {
    float a = x.v.x, b = x.v.y;
    a = a < -87.3f ? -87.3f : a;
    a = a > 89.0f ? 89.0f : a;
    b = b < -87.3f ? -87.3f : b;
    b = b > 89.0f ? 89.0f : b;
    const f32x2 xc(a, b);
    const f32x2 kx = xc * f32x2(1.44269504088896341f);
    const float ka = rintf(kx.v.x), kb = rintf(kx.v.y);
    const f32x2 nk(-ka, -kb);
    f32x2 r = fma(nk, f32x2(0.693145751953125f), xc);
    r = fma(nk, f32x2(1.42860682030941723e-6f), r);
    f32x2 q(1.0f / 40320.0f);
    q = fma(q, r, f32x2(1.0f / 5040.0f));
    q = fma(q, r, f32x2(1.0f / 720.0f));
    q = fma(q, r, f32x2(1.0f / 120.0f));
    q = fma(q, r, f32x2(1.0f / 24.0f));
    q = fma(q, r, f32x2(1.0f / 6.0f));
    q = fma(q, r, f32x2(0.5f));
    const f32x2 e = fma(q, r * r, r);
    const f32x2 t(__int_as_float(((int)ka + 127) << 23), __int_as_float(((int)kb + 127) << 23));
    return fma(t, e, t - f32x2(1.0f));
}

__device__ __forceinline__ void sincos_small(double x, double* s, double* c) {
    if (small_arg(x)) {
        double t = x * x;
        double ps = 1.0 / 5040.0;  // sin(x)/x = 1 - t/6 + t^2/120 - t^3/5040
        ps = fma(ps, -t, 1.0 / 120.0);
        ps = fma(ps, -t, 1.0 / 6.0);
        ps = fma(ps, -t, 1.0);
        *s = ps * x;
        double pc = 1.0 / 720.0;  // cos(x) = 1 - t/2 + t^2/24 - t^3/720
        pc = fma(pc, -t, 1.0 / 24.0);
        pc = fma(pc, -t, 0.5);
        *c = fma(pc, -t, 1.0);
        return;
    }
    sincos(x, s, c);
}
__device__ __forceinline__ void sincos_small(float x, float* s, float* c) { sincosf(x, s, c); }


// Coefficients of exp(-z A) = I - s_z A + k_z A^2 for the HERM matrix A
// (A^3 = C^2 A since A has eigenvalues C, 0, -C):
//   imaginary time (z = dt):  s = sinh(dt C)/C,  k = (cosh(dt C) - 1)/C^2
//   real time (z = i dt):     s_z = i s, s = sin(dt C)/C,  k = (cos(dt C) - 1)/C^2
// Both are even in C, so for small w = (dt C)^2 they are power series in w:
//   s = dt  sum_n (+-w)^n/(2n+1)!,   k = +-dt^2 sum_n (+-w)^n/(2n+2)!
// (+ for imaginary, - for real time); no square root is needed. Otherwise
// C = sqrt(C^2) and the closed forms, with cosh - 1 = 2 sinh^2(x/2) and
// cos - 1 = -2 sin^2(x/2) to avoid cancellation.
template <bool IMAG>
__device__ __forceinline__ void herm_coeffs(double C2, double dt, double* s, double* k) {
    double w = dt * dt * C2;  // >= 0
    if ((unsigned)__double2hiint(w) < 0x3EB00000u) {
        // w < 2^-20: three terms each (first omitted terms < 2e-22 relative)
        double v = IMAG ? w : -w;
        double ps = fma(fma(v, 1.0 / 120.0, 1.0 / 6.0), v, 1.0);
        double pk = fma(fma(v, 1.0 / 720.0, 1.0 / 24.0), v, 0.5);
        *s = dt * ps;
        *k = (IMAG ? dt * dt : -dt * dt) * pk;
        return;
    }
    if (w <= 1.0 / 1024.0) {
        double v = IMAG ? w : -w;
        double ps = 1.0 / 362880.0;  // 1/9!
        ps = fma(ps, v, 1.0 / 5040.0);
        ps = fma(ps, v, 1.0 / 120.0);
        ps = fma(ps, v, 1.0 / 6.0);
        ps = fma(ps, v, 1.0);
        double pk = 1.0 / 3628800.0;  // 1/10!
        pk = fma(pk, v, 1.0 / 40320.0);
        pk = fma(pk, v, 1.0 / 720.0);
        pk = fma(pk, v, 1.0 / 24.0);
        pk = fma(pk, v, 0.5);
        *s = dt * ps;
        *k = (IMAG ? dt * dt : -dt * dt) * pk;
        return;
    }
    double C = sqrt(C2);
    double x = dt * C;
    if (IMAG) {
        double sh = sinh(0.5 * x);
        *s = sinh(x) / C;
        *k = 2.0 * sh * sh / C2;
    } else {
        double sh = sin(0.5 * x);
        *s = sin(x) / C;
        *k = -2.0 * sh * sh / C2;
    }
}
template <bool IMAG>
__device__ __forceinline__ void herm_coeffs(float C2, float dt, float* s, float* k) {
    float w = dt * dt * C2;
    if (w <= 1.0f / 256.0f) {
        float v = IMAG ? w : -w;
        float ps = fmaf(fmaf(1.0f / 5040.0f, v, 1.0f / 120.0f), v, 1.0f / 6.0f);
        ps = fmaf(ps, v, 1.0f);
        float pk = fmaf(fmaf(1.0f / 40320.0f, v, 1.0f / 720.0f), v, 1.0f / 24.0f);
        pk = fmaf(pk, v, 0.5f);
        *s = dt * ps;
        *k = (IMAG ? dt * dt : -dt * dt) * pk;
        return;
    }
    float C = sqrtf(C2);
    float x = dt * C;
    if (IMAG) {
        float sh = sinhf(0.5f * x);
        *s = sinhf(x) / C;
        *k = 2.0f * sh * sh / C2;
    } else {
        float sh = sinf(0.5f * x);
        *s = sinf(x) / C;
        *k = -2.0f * sh * sh / C2;
    }
}

// herm_coeffs on a pair of points: the series on the packed instructions when
// both lanes are in its range, otherwise lane by lane.
template <bool IMAG>
__device__ __forceinline__ void herm_coeffs_pair(f32x2 C2, f32x2 dt, f32x2* s, f32x2* k) {
    const f32x2 w = dt * dt * C2;
    if (w.v.x <= 1.0f / 256.0f && w.v.y <= 1.0f / 256.0f) {
        const f32x2 v = IMAG ? w : -w;
        f32x2 ps = fma(fma(f32x2(1.0f / 5040.0f), v, f32x2(1.0f / 120.0f)), v, f32x2(1.0f / 6.0f));
        ps = fma(ps, v, f32x2(1.0f));
        f32x2 pk = fma(fma(f32x2(1.0f / 40320.0f), v, f32x2(1.0f / 720.0f)), v, f32x2(1.0f / 24.0f));
        pk = fma(pk, v, f32x2(0.5f));
        *s = dt * ps;
        *k = (IMAG ? dt * dt : -dt * dt) * pk;
        return;
    }
    float s0, k0, s1, k1;
    herm_coeffs<IMAG>(C2.v.x, dt.v.x, &s0, &k0);
    herm_coeffs<IMAG>(C2.v.y, dt.v.y, &s1, &k1);
    *s = f32x2(s0, s1);
    *k = f32x2(k0, k1);
}

// Multiply by z/dt: 1 in imaginary time, i in real time.
template <bool IMAG, typename R> __device__ __forceinline__ cx<R> zunit(cx<R> a) {
    if (IMAG) return a;
    return {-a.im, a.re};
}

// ---------------------------------------------------------------------------
// Kernel parameter block (host-computed constants; plain data).
// ---------------------------------------------------------------------------
struct KParams {
    int dim, nx, ny;
    int so_case;      // 0 none; 1 1D Sigma_x; 2 1D Sigma_y; 3 1D Sigma_z; 4 2D (eta)
    double dx, dy, dt;
    double hx, hy;    // SO: dt*gt/(2dx) (dt*gamma/(2dx) for Sigma_z), dt*gt*eta/(2dy)
    double sx, sy;    // the same without the factor dt (for the SO energy)
    double c0, c2;
    double wx2h, wy2h;  // wx^2/2, wy^2/2
    double vx, vy;      // wx^2 dx^2/2, wy^2 dy^2/2 (trap per squared grid index)
    double omega_t;   // Omega/sqrt2 (constant Rabi term)
    double wx, wy;    // trap frequencies (for the trap gradient of the adjoint)
    double cell;      // dx (1D) or dx*dy
    int renorm;       // 0, 1 (DJ2), 2 (DJ)
    double mag;
    int split, so_mode;  // Strang splitting, SO by Crank-Nicolson (sgpe_params)
    // Constants of the pointwise substeps in each arithmetic type (kc<R>):
    // kd the FP64 value, kf its FP32 rounding, kl the FP32 rest kd - kf (the
    // double-float low part); filled by fill_derived on the host before a
    // launch, so no kernel converts a constant per grid point.
    double kd[32];
    float kf[32], kl[32];
};

// Indices into KParams::kd / kf / kl. NC0..NVY: -dt times c0, c2, vx, vy (dt
// folded into the CALCNU exponent); HS0 + n, HK0 + n: the HERM series
// coefficients dt/(2n+1)! and dt^2/(2n+2)!, n = 0..4.
enum KC {
    KC_DT, KC_HX, KC_HY, KC_C0, KC_C2, KC_VX, KC_VY, KC_OMEGA,
    KC_NC0, KC_NC2, KC_NVX, KC_NVY, KC_DT2, KC_HS0, KC_HK0 = KC_HS0 + 5, KC_N = KC_HK0 + 5
};
static_assert(KC_N <= 32, "KParams constant table too small");

inline void fill_derived(KParams& k) {
    double* d = k.kd;
    d[KC_DT] = k.dt;
    d[KC_HX] = k.hx;
    d[KC_HY] = k.hy;
    d[KC_C0] = k.c0;
    d[KC_C2] = k.c2;
    d[KC_VX] = k.vx;
    d[KC_VY] = k.vy;
    d[KC_OMEGA] = k.omega_t;
    d[KC_NC0] = -k.dt * k.c0;
    d[KC_NC2] = -k.dt * k.c2;
    d[KC_NVX] = -k.dt * k.vx;
    d[KC_NVY] = -k.dt * k.vy;
    d[KC_DT2] = k.dt * k.dt;
    double f = 1.0;  // (2n+1)!
    for (int n = 0; n < 5; n++) {
        if (n > 0) f *= (2.0 * n) * (2.0 * n + 1.0);
        d[KC_HS0 + n] = k.dt / f;
        d[KC_HK0 + n] = d[KC_DT2] / (f * (2.0 * n + 2.0));
    }
    for (int i = 0; i < KC_N; i++) {
        k.kf[i] = (float)d[i];
        k.kl[i] = (float)(d[i] - (double)k.kf[i]);
    }
}

// Constant i of the pointwise substeps in the arithmetic type R.
// Lines longer than 1024 points: 16 points a lane, at most 16 warps a block.
constexpr int kLongC = 16;
constexpr int kLongMaxWarps = 16;
// Row tiles of the y sweep of long columns (k_cn_y_tile): chunks of kLongC rows
// a tile writes, the most halo chunks above and below, rows written per tile.
// (kTileReal: the tall tiles; grids of at most kTileShortMaxN rows take tiles of
// kTileRealShort chunks, which gives short columns more tiles)
constexpr int kTileReal = 8, kTileMaxHalo = 2;
constexpr int kTileRealShort = 4, kTileShortMaxN = 512;
constexpr int kTileMaxWarps = kTileReal + 2 * kTileMaxHalo;
constexpr int kTileRows = kLongC * kTileReal;
// Extra elements between the staged columns of a y tile of lines longer than
// 1024 points (complex64 tiles of 4 columns; see k_cn_y).
__host__ __device__ constexpr int long_col_pad(int elem_bytes, int kc) { return (elem_bytes == 8 && kc == 4) ? 4 : 0; }

template <typename R> __device__ __forceinline__ R kc(const KParams& p, int i);
template <> __device__ __forceinline__ double kc<double>(const KParams& p, int i) { return p.kd[i]; }
template <> __device__ __forceinline__ float kc<float>(const KParams& p, int i) { return p.kf[i]; }
template <> __device__ __forceinline__ df kc<df>(const KParams& p, int i) { return df(p.kf[i], p.kl[i]); }
template <> __device__ __forceinline__ f32x2 kc<f32x2>(const KParams& p, int i) { return f32x2(p.kf[i]); }

// Programmatic dependent launch (sm_90+). The step kernels are launched with
// programmatic stream serialization, so a kernel's blocks may be scheduled
// while its predecessor on the stream is still running: every such kernel
// first lets its own successor launch (pdl_trigger), then waits until the
// predecessor grid has completed and its writes are visible (pdl_wait) before
// it touches any data the predecessor produces. Launched normally, both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


// ---------------------------------------------------------------------------
// Pointwise substeps at one grid point. u[j] holds the (already scaled) state
// of component j at the point; X[j], Y[j] the raw differences
// psi_j(x+1) - psi_j(x-1), psi_j(y+1) - psi_j(y-1) with zero ghosts, and d[j]
// the scale of component j (the pending renormalisation).
// ---------------------------------------------------------------------------

// SO (Appendix A Eqs. (p1)-(p2)): u_j <- u_j - z (H_SO psi)_j, with H_SO from
// the SO terms of Sec. 2 (1D Sigma_y in the form derived from gamma p_x Sigma_y).
template <bool IMAG, typename R>
__device__ __forceinline__ void so_point(cx<R> (&u)[3], const cx<R> (&X)[3], const cx<R> (&Y)[3],
                                         const R (&gx)[3], const R (&gy)[3], int so_case) {
    // h'_j = dt * (H_SO psi)_j; the update is u_j -= zunit(h'_j).
    cx<R> h0, hp, hm;
    if (so_case == 4) {
        // f_+ = gt d_x psi_0 - i gt eta d_y psi_0 ; f_- = -gt d_x psi_0 - i gt eta d_y psi_0
        // g = -gt d_x psi_+ + gt d_x psi_- - i gt eta d_y (psi_+ + psi_-)
        cx<R> ax = scl(gx[1], X[1]);
        cx<R> ay = {gy[1] * Y[1].im, -gy[1] * Y[1].re};  // -i gy Y0
        hp = add(ax, ay);
        hm = sub(ay, ax);
        h0.re = fma(-gx[0], X[0].re, fma(gx[2], X[2].re, fma(gy[0], Y[0].im, gy[2] * Y[2].im)));
        h0.im = fma(-gx[0], X[0].im, fma(gx[2], X[2].im, -fma(gy[0], Y[0].re, gy[2] * Y[2].re)));
    } else if (so_case == 1) {
        // Sigma_x: f_+- = -i gt d_x psi_0 ; g = -i gt d_x (psi_+ + psi_-)
        hp = {gx[1] * X[1].im, -gx[1] * X[1].re};
        hm = hp;
        h0.re = fma(gx[0], X[0].im, gx[2] * X[2].im);
        h0.im = -fma(gx[0], X[0].re, gx[2] * X[2].re);
    } else if (so_case == 2) {
        // Sigma_y: f_+ = -gt d_x psi_0 ; f_- = gt d_x psi_0 ; g = gt d_x (psi_+ - psi_-)
        hm = scl(gx[1], X[1]);
        hp = {-hm.re, -hm.im};
        h0.re = fma(gx[0], X[0].re, -gx[2] * X[2].re);
        h0.im = fma(gx[0], X[0].im, -gx[2] * X[2].im);
    } else if (so_case == 3) {
        // Sigma_z: f_+ = -i gamma d_x psi_+ ; f_- = +i gamma d_x psi_- ; g = 0
        hp = {gx[0] * X[0].im, -gx[0] * X[0].re};
        hm = {-gx[2] * X[2].im, gx[2] * X[2].re};
        h0 = {R(0), R(0)};
    } else {
        return;
    }
    u[0] = sub(u[0], zunit<IMAG>(hp));
    u[1] = sub(u[1], zunit<IMAG>(h0));
    u[2] = sub(u[2], zunit<IMAG>(hm));
}

// CALCNU: u_j <- exp(-z mu_j) u_j with
//   mu_+- = V + c0 rho + c2 (rho_+- - rho_-+ + rho_0),  mu_0 = V + c0 rho + c2 (rho_+ + rho_-).
template <bool IMAG, typename R>
__device__ __forceinline__ void calcnu_point(cx<R> (&u)[3], R V, R c0, R c2, R dt) {
    R rp = nrm(u[0]), r0 = nrm(u[1]), rm = nrm(u[2]);
    R base = fma(c0, rp + r0 + rm, V);
    R mup = fma(c2, rp - rm + r0, base);
    R mu0 = fma(c2, rp + rm, base);
    R mum = fma(c2, rm - rp + r0, base);
    if constexpr (is_pair<R>()) {
        // the complex64 form below on a pair of points
        const R mu[3] = {mup, mu0, mum};
        const R ndt = -dt, hdt = R(0.5f) * dt;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (IMAG) {
                u[j] = axpy(expm1_cw(ndt * mu[j]), u[j], u[j]);
            } else {
                const R t = hdt * mu[j];
                float s0, c0_, s1, c1_;
                sincosf(t.v.x, &s0, &c0_);
                sincosf(t.v.y, &s1, &c1_);
                const R sh(s0, s1), ch(c0_, c1_), m2 = R(-2.0f) * sh;
                const cx<R> fm1 = {m2 * sh, m2 * ch};  // exp(-i t) - 1
                u[j] = add(u[j], mul(fm1, u[j]));
            }
        }
    } else if constexpr (sizeof(R) == 4) {
        // complex64 state: apply the factor as u + (f - 1) u with f - 1 formed
        // without cancellation, so that rounding the factor cannot bias |u|
        // the same way every step (expm1; cos t - 1 = -2 sin^2(t/2)).
        const R mu[3] = {mup, mu0, mum};
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (IMAG) {
                u[j] = axpy((R)expm1_cw((float)(-dt * mu[j])), u[j], u[j]);
            } else {
                float sh, ch;
                sincosf((float)(0.5f * dt * mu[j]), &sh, &ch);
                const cx<R> fm1 = {(R)(-2.0f * sh * sh), (R)(-2.0f * sh * ch)};  // exp(-i t) - 1
                u[j] = add(u[j], mul(fm1, u[j]));
            }
        }
    } else if (IMAG) {
        R fp = exp_small(-dt * mup), f0 = exp_small(-dt * mu0), fm = exp_small(-dt * mum);
        u[0] = scl(fp, u[0]);
        u[1] = scl(f0, u[1]);
        u[2] = scl(fm, u[2]);
    } else {
        R s, c;
        sincos_small(dt * mup, &s, &c);  // exp(-i dt mu) = c - i s
        u[0] = mul(cx<R>{c, -s}, u[0]);
        sincos_small(dt * mu0, &s, &c);
        u[1] = mul(cx<R>{c, -s}, u[1]);
        sincos_small(dt * mum, &s, &c);
        u[2] = mul(cx<R>{c, -s}, u[2]);
    }
}

// CALCNU for the complex128 state with dt folded into the coefficients
// (KParams::n_*): Vn = -dt V, exponents x_j = -dt mu_j; imaginary time
// u_j <- exp(x_j) u_j, real time u_j <- (cos x_j + i sin x_j) u_j = exp(-i dt mu_j) u_j.
template <bool IMAG, typename R>
__device__ __forceinline__ void calcnu_point_dt(cx<R> (&u)[3], R Vn, const KParams& p) {
    R rp = nrm(u[0]), r0 = nrm(u[1]), rm = nrm(u[2]);
    const R nc0 = kc<R>(p, KC_NC0), nc2 = kc<R>(p, KC_NC2);
    R base = fma(nc0, rp + r0 + rm, Vn);
    R x[3] = {fma(nc2, rp - rm + r0, base), fma(nc2, rp + rm, base), fma(nc2, rm - rp + r0, base)};
#pragma unroll
    for (int j = 0; j < 3; j++) {
        if (IMAG) {
            u[j] = scl(exp_small(x[j]), u[j]);
        } else {
            R s, c;
            sincos_small(x[j], &s, &c);
            u[j] = mul(cx<R>{c, s}, u[j]);
        }
    }
}

// HERM coefficients s, k (see herm_coeffs) from the dt-folded series constants
// KParams::hs, hk: s = sum_n hs_n v^n, k = +-sum_n hk_n v^n, v = +-dt^2 C^2.
// w = dt^2 C^2 against 2^-20 and 1/1024 (the series ranges below).
__device__ __forceinline__ bool w_tiny(double w) { return (unsigned)__double2hiint(w) < 0x3EB00000u; }
__device__ __forceinline__ bool w_tiny(df w) { return w.hi < 9.5367431640625e-07f; }
__device__ __forceinline__ bool w_small(double w) { return w <= 1.0 / 1024.0; }
__device__ __forceinline__ bool w_small(df w) { return w.hi <= 1.0f / 1024.0f; }

template <bool IMAG, typename R>
__device__ __forceinline__ void herm_coeffs_dt(R C2, const KParams& p, R* s, R* k) {
    R w = kc<R>(p, KC_DT2) * C2;  // >= 0
    R v = IMAG ? w : -w;
    if (w_tiny(w)) {
        // w < 2^-20: three terms each
        *s = fma(fma(v, kc<R>(p, KC_HS0 + 2), kc<R>(p, KC_HS0 + 1)), v, kc<R>(p, KC_HS0));
        R pk = fma(fma(v, kc<R>(p, KC_HK0 + 2), kc<R>(p, KC_HK0 + 1)), v, kc<R>(p, KC_HK0));
        *k = IMAG ? pk : -pk;
        return;
    }
    if (w_small(w)) {
        R ps = kc<R>(p, KC_HS0 + 4), pk = kc<R>(p, KC_HK0 + 4);
#pragma unroll
        for (int n = 3; n >= 0; n--) {
            ps = fma(ps, v, kc<R>(p, KC_HS0 + n));
            pk = fma(pk, v, kc<R>(p, KC_HK0 + n));
        }
        *s = ps;
        *k = IMAG ? pk : -pk;
        return;
    }
    // rare: closed forms in FP64
    double sd, kd;
    herm_coeffs<IMAG>(dbl(C2), p.dt, &sd, &kd);
    *s = to_r<R>(sd);
    *k = to_r<R>(kd);
}

// HERM (Appendix A): with a = c2 psi_-^* psi_0 + Ot, b = c2 psi_0^* psi_+ + Ot
// and A = [[0,a,0],[a*,0,b],[0,b*,0]] (frozen over the substep), psi <- exp(-z A) psi,
// evaluated as psi - s_z A psi + k A^2 psi with A^2 = [[|a|^2,0,ab],[0,C^2,0],[a*b*,0,|b|^2]].
// This equals the eigen-decomposition form V diag(exp(-z lambda)) V^{-1} of Eq. (11) and
// stays finite at C = 0.
// kp: the kernel constants (complex128 and double-float take s, k from the
// dt-folded series constants; complex64 evaluates them from dt).
template <bool IMAG, typename R>
__device__ __forceinline__ void herm_point(cx<R> (&u)[3], R c2, R Ot, R dt, const KParams* kp) {
    cx<R> a = cmul(u[2], u[1]);  // psi_-^* psi_0
    a = {fma(c2, a.re, Ot), c2 * a.im};
    cx<R> b = cmul(u[1], u[0]);  // psi_0^* psi_+
    b = {fma(c2, b.re, Ot), c2 * b.im};
    R na = nrm(a), nb = nrm(b);
    R C2 = na + nb;
    R s, k;
    if constexpr (is_pair<R>()) {
        herm_coeffs_pair<IMAG>(C2, dt, &s, &k);
    } else if constexpr (is_f32<R>()) {
        herm_coeffs<IMAG>(C2, dt, &s, &k);
    } else {
        herm_coeffs_dt<IMAG>(C2, *kp, &s, &k);
    }
    cx<R> ab = mul(a, b);
    // A psi
    cx<R> Ap = mul(a, u[1]);
    cx<R> A0 = add(cmul(a, u[0]), mul(b, u[2]));
    cx<R> Am = cmul(b, u[1]);
    // A^2 psi
    cx<R> Bp = axpy(na, u[0], mul(ab, u[2]));
    cx<R> B0 = scl(C2, u[1]);
    cx<R> Bm = axpy(nb, u[2], cmul(ab, u[0]));
    cx<R> sAp = zunit<IMAG>(Ap), sA0 = zunit<IMAG>(A0), sAm = zunit<IMAG>(Am);
    u[0] = axpy(k, Bp, axpy(-s, sAp, u[0]));
    u[1] = axpy(k, B0, axpy(-s, sA0, u[1]));
    u[2] = axpy(k, Bm, axpy(-s, sAm, u[2]));
}

// HERM for the double-float state. The update psi - s_z A psi + k A^2 psi has
// terms of sizes ~ dt C |psi| and ~ (dt C)^2 |psi| / 2. When w = (dt C)^2 <
// 2^-25, the second term and the series corrections of s and k are formed in
// FP32 from the leading parts (their FP32 rounding stays below 2^-50 |psi| and
// the dropped series terms below 2^-57 |psi|); the A psi term and the updates
// stay in double-float. Otherwise the general double-float evaluation.
template <bool IMAG>
__device__ __forceinline__ void herm_point_df(cx<df> (&u)[3], df c2, df Ot, const KParams& p) {
    cx<df> a = cmul(u[2], u[1]);  // psi_-^* psi_0
    a = {fma(c2, a.re, Ot), c2 * a.im};
    cx<df> b = cmul(u[1], u[0]);  // psi_0^* psi_+
    b = {fma(c2, b.re, Ot), c2 * b.im};
    const float ar = a.re.hi, ai = a.im.hi, br = b.re.hi, bi = b.im.hi;
    const float na = fmaf(ar, ar, ai * ai), nb = fmaf(br, br, bi * bi), C2 = na + nb;
    const float w = p.kf[KC_DT2] * C2;
    if (!(w < 2.98023223876953125e-08f)) {
        // general case: every term in double-float
        df na_d = nrm(a), nb_d = nrm(b), C2_d = na_d + nb_d, s, k;
        herm_coeffs_dt<IMAG>(C2_d, p, &s, &k);
        cx<df> ab = mul(a, b);
        cx<df> Ap = mul(a, u[1]), A0 = add(cmul(a, u[0]), mul(b, u[2])), Am = cmul(b, u[1]);
        cx<df> Bp = axpy(na_d, u[0], mul(ab, u[2])), B0 = scl(C2_d, u[1]), Bm = axpy(nb_d, u[2], cmul(ab, u[0]));
        u[0] = axpy(k, Bp, axpy(-s, zunit<IMAG>(Ap), u[0]));
        u[1] = axpy(k, B0, axpy(-s, zunit<IMAG>(A0), u[1]));
        u[2] = axpy(k, Bm, axpy(-s, zunit<IMAG>(Am), u[2]));
        return;
    }
    const float v = IMAG ? w : -w;
    // s = dt (1 + v/6 + ...), k = +-dt^2 (1/2 + v/24 + ...)
    const df s = add_f(kc<df>(p, KC_HS0), p.kf[KC_HS0 + 1] * v);
    const float kk = fmaf(p.kf[KC_HK0 + 1], v, p.kf[KC_HK0]);
    const float k = IMAG ? kk : -kk;
    // A psi (double-float)
    const cx<df> Ap = mul(a, u[1]);
    const cx<df> A0 = add(cmul(a, u[0]), mul(b, u[2]));
    const cx<df> Am = cmul(b, u[1]);
    // k A^2 psi (FP32, leading parts)
    const cx<float> a_f = {ar, ai}, b_f = {br, bi};
    const cx<float> u0 = {u[0].re.hi, u[0].im.hi}, u1 = {u[1].re.hi, u[1].im.hi}, u2 = {u[2].re.hi, u[2].im.hi};
    const cx<float> ab = mul(a_f, b_f);
    const cx<float> Bp = scl(k, axpy(na, u0, mul(ab, u2)));
    const cx<float> B0 = scl(k * C2, u1);
    const cx<float> Bm = scl(k, axpy(nb, u2, cmul(ab, u0)));
    const cx<df> sAp = zunit<IMAG>(Ap), sA0 = zunit<IMAG>(A0), sAm = zunit<IMAG>(Am);
    u[0] = {add_f(u[0].re - s * sAp.re, Bp.re), add_f(u[0].im - s * sAp.im, Bp.im)};
    u[1] = {add_f(u[1].re - s * sA0.re, B0.re), add_f(u[1].im - s * sA0.im, B0.im)};
    u[2] = {add_f(u[2].re - s * sAm.re, Bm.re), add_f(u[2].im - s * sAm.im, Bm.im)};
}

}  // namespace sgpe
