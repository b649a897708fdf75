// sgpe_kernels.cuh -- sm_103a kernels of one split step (arXiv:2009.13507,
// Sec. 3 and Appendix A) for one grid, templated on the storage precision R
// (double: complex128 state; float: complex64 state) and on the time mode
// (IMAG: z = dt, imaginary time; otherwise z = i dt, real time).
//
// One step, 2D with lines of at most 1024 points (sgpe_cn.cuh):
//   k_pwx      (A -> B): pending scale, SO, CALCNU, HERM, then Crank-Nicolson
//                        along x from shared memory, one block per row
//   k_cny_reg  (B -> A): Crank-Nicolson along y, one warp per column (pair),
//                        FP64 norm partials
//   k_finalize         : norms, next pending scale, step counter
// Longer lines: k_pointwise and the shared-memory sweeps k_cn_x / k_cn_y below.
// One step, 1D: k_pointwise (A -> B), the x sweep (B -> A) with norm partials,
// k_finalize.
// Reductions are FP64 in both precisions and deterministic (fixed order).
#pragma once
#include <type_traits>

#include "sgpe_device.cuh"

namespace sgpe {

// ---------------------------------------------------------------------------
// Workspace scalars (device) used by the step kernels.
// ---------------------------------------------------------------------------
struct DevScalars {
    double scale[4];     // pending renormalisation scale per component (DJ2: all equal)
    float scale_f[4];    // the same rounded to FP32 (read by the complex64 form)
    float scale_l[4];    // and the rest scale - scale_f (double-float low part)
    int scale_src;       // 1: the pending scale is still to be derived from the last y sweep's
                         // norm partials (the fused 2D step); 0: scale[] holds it
    double norms[4];     // N_j of the state written by the last completed step
    double obs[16];      // observables of the last sgpe_energy
    int step_idx;        // index into a per-step Omega table (real time)
    int err;             // bit 0: non-finite norm
    unsigned ticket[4];  // last-block tickets: 0 step finalize, 1 observables, 2 norms
};

// Crank-Nicolson coefficient tables for one axis and one time mode.
// T = I - bt L (L = tridiag(1,-2,1), bt = z/(4h^2)) factors as T = L U with
// u_0 = 1 + 2bt, u_i = 1 + 2bt - bt^2/u_{i-1}. With y'_i = y_i/u_i:
//   forward  y'_i = fa_i x_i + fg_i y'_{i-1},  fa_i = 1/u_i, fg_i = bt/u_i
//   backward w_i  = y'_i + fg_i w_{i+1}
// and the step's Crank-Nicolson result is 2 w - x  (= T^{-1}(I + bt L) x).
// A warp solves a line in 32 chunks of C consecutive points; fp_i / fq_i are the
// products of fg over the chunk up to / from point i (carry propagation).
//
// Lines longer than 1024 points with uks > 0 skip the tables. The pivots u_i
// converge to the root u of u^2 - (1 + 2bt) u + bt^2 = 0 with |u| > |bt| (a
// contraction: |bt/u|^2 < 1). T' = T with its first diagonal entry replaced by u
// has the constant factors ua = 1/u, ug = bt/u at every point; T = T' + delta
// e_0 e_0^T with delta = 1 + 2bt - u, so (Sherman-Morrison) T^{-1} r = w - uc w_0 s
// with w = T'^{-1} r, s = T'^{-1} e_0 and uc = delta / (1 + delta s_0). s decays
// like ug^i: its first uks entries (us) are the ones above 2^-64 / |uc|. unlev:
// carry-scan levels after which the composed chunk factor ug^(16 2^L) is below
// 2^-64 (the cut of tiny_carry). uk: the factor that turns the solve's scaled
// unknown q = w / ua into the sweep's result (2 ua for 2w - x, 2 bt ua for the
// increment form x + 2e). upow[k] = ug^(k+1), k < 16 (imaginary time: the
// real power in both halves), the chunk carry weights.
template <typename R> struct Tabs {
    const typename V2<R>::T* fa;
    const typename V2<R>::T* fg;
    const typename V2<R>::T* fp;
    const typename V2<R>::T* fq;
    cx<R> ug, ug16, uc, uk;
    cx<R> upow[16];
    const typename V2<R>::T* us;
    int uks, unlev;
};


template <bool IMAG, typename R> __device__ __forceinline__ cx<R> tmul(cx<R> t, cx<R> x) {
    if (IMAG) return scl(t.re, x);
    return mul(t, x);
}
// acc + t * x
template <bool IMAG, typename R> __device__ __forceinline__ cx<R> tfma(cx<R> t, cx<R> x, cx<R> acc) {
    if (IMAG) return axpy(t.re, x, acc);
    return caxpy(t, x, acc);
}
__device__ __forceinline__ double shfl_up_r(double v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
__device__ __forceinline__ float shfl_up_r(float v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
__device__ __forceinline__ df shfl_up_r(df v, int off) {
    return df(__shfl_up_sync(0xffffffffu, v.hi, off), __shfl_up_sync(0xffffffffu, v.lo, off));
}
__device__ __forceinline__ double shfl_dn_r(double v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
__device__ __forceinline__ float shfl_dn_r(float v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
__device__ __forceinline__ df shfl_dn_r(df v, int off) {
    return df(__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off));
}
template <typename R> __device__ __forceinline__ cx<R> shup(cx<R> a, int off) {
    return {shfl_up_r(a.re, off), shfl_up_r(a.im, off)};
}
template <typename R> __device__ __forceinline__ cx<R> shdn(cx<R> a, int off) {
    return {shfl_dn_r(a.re, off), shfl_dn_r(a.im, off)};
}

// Early end of the lanes' carry scans. After the scan level with offset off,
// lane l holds the composed chunk map of lanes [l - 2 off + 1, l] (forward) or
// [l, l + 2 off - 1] (backward); every further level only adds terms weighted
// by that map's factor A times more chunk factors. The CN matrix is strictly
// diagonally dominant, so every LU ratio fg has |fg| < 1 and so has every
// chunk factor; once each lane's |A| < 2^-64 (or its window already reaches
// the line's end) the remaining terms are below 2^-59 of the line's largest
// value, far below its rounding, and the scan stops. For small bt (the usual
// case: bt = dt/(4 h^2) ~ 0.02 gives |fg| ~ 0.02 and, with 8-point chunks, a
// chunk factor ~ 2^-46) one level suffices instead of five. The test reads
// the exponent on the integer pipe (FP64 compares would cost FP64 issue slots).
// Complex128 only: there each skipped level saves FP64 instructions; the
// complex64 and double-float scans run on the FP32 pipe, where the vote and
// its register pressure measured slower than the full scan.
__device__ __forceinline__ bool tiny_carry(double x) {
    return ((unsigned)__double2hiint(x) & 0x7fffffffu) < 0x3BF00000u;  // |x| < 2^-64
}
// (also used, in every precision, to cut the composition of the warps' segment
// maps of lines longer than 1024 points)
__device__ __forceinline__ bool tiny_carry(float x) { return fabsf(x) < 5.42101086242752217e-20f; }
__device__ __forceinline__ bool tiny_carry(df x) { return fabsf(x.hi) < 5.42101086242752217e-20f; }
// Whether every lane of the warp is done after a level: edge (its window
// reaches the line's end) or a negligible composed factor A.
template <typename R> __device__ __forceinline__ bool scan_done(bool edge, const cx<R>& A) {
    if constexpr (std::is_same<R, double>::value)
        return __all_sync(0xffffffffu, edge || (tiny_carry(A.re) && tiny_carry(A.im)));
    else
        return false;
}

template <typename R> __device__ __forceinline__ cx<R> tld(const typename V2<R>::T* t, int i) {
    return unpack(__ldg(t + i));
}

// Deterministic block reduction of NV doubles per thread; result valid in
// thread 0. red: shared scratch of (blockDim/32)*NV doubles.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) red[warp * NV + q] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double s = 0.0;
            for (int w = 0; w < nw; w++) s += red[w * NV + q];
            v[q] = s;
        }
    }
}

// Last-block election after every block wrote its partials; returns true in
// all threads of the last block to arrive (threadfence-reduction pattern).
__device__ __forceinline__ bool last_block(unsigned* ticket) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == nb - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// Renormalisation factors from the norms (Appendix A): Eq. (DJ2) for renorm = 1,
// Eq. (DJ) with magnetisation mag for renorm = 2; otherwise 1.
__device__ __forceinline__ void renorm_factors(const double (&N)[3], int renorm, double mag, double (&d)[3]) {
    d[0] = d[1] = d[2] = 1.0;
    if (!(N[0] + N[1] + N[2] > 0.0)) return;  // a zero state has no normalisation: left as it is
    if (renorm == 1) {
        double f = rsqrt(N[0] + N[1] + N[2]);  // one reciprocal square root: a short FP64 chain
        d[0] = d[1] = d[2] = f;
    } else if (renorm == 2) {
        double m = mag;
        double den = N[1] + sqrt(4.0 * (1.0 - m * m) * N[0] * N[2] + m * m * N[1] * N[1]);
        if (!(den > 0.0)) return;
        double d0 = sqrt(1.0 - m * m) / sqrt(den);
        d[0] = N[0] > 0.0 ? sqrt(1.0 + m - d0 * d0 * N[1]) / sqrt(2.0 * N[0]) : 1.0;
        d[2] = N[2] > 0.0 ? sqrt(1.0 - m - d0 * d0 * N[1]) / sqrt(2.0 * N[2]) : 1.0;
        d[1] = N[1] > 0.0 ? d0 : 1.0;
    }
}

// Called by every thread of the last block: sum the per-block partial norms
// (partials[b*3 + j]) in block order, then thread 0 publishes N_j, the next
// pending scale (renorm != 0) and advances the step counter.
__device__ __forceinline__ void finalize_norms(const double* partials, int nblk, double cell, int renorm,
                                               double mag, bool advance_step, DevScalars* sc, unsigned* ticket) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double s[3] = {0.0, 0.0, 0.0};
        for (int b = lane; b < nblk; b += 32) {
            s[0] += __ldcg(partials + 3 * b + 0);
            s[1] += __ldcg(partials + 3 * b + 1);
            s[2] += __ldcg(partials + 3 * b + 2);
        }
#pragma unroll
        for (int q = 0; q < 3; q++)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
        if (lane == 0) {
            double N[3] = {s[0] * cell, s[1] * cell, s[2] * cell};
            bool finite = isfinite(N[0]) && isfinite(N[1]) && isfinite(N[2]);
            double d[3];
            renorm_factors(N, finite ? renorm : 0, mag, d);
            for (int j = 0; j < 3; j++) {
                sc->norms[j] = N[j];
                sc->scale[j] = d[j];
                sc->scale_f[j] = (float)d[j];
                sc->scale_l[j] = (float)(d[j] - (double)sc->scale_f[j]);
            }
            if (!finite) sc->err |= 1;
            if (advance_step) sc->step_idx += 1;
            sc->scale_src = 0;
            *ticket = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Pointwise substeps (SO, CALCNU, HERM) of one step; mask selects substeps
// (bit 0 SO, bit 1 CALCNU, bit 2 HERM) and how: bit 3 (kMaskReverse) HERM
// before CALCNU (the second half of a Strang step), bit 4 (kMaskNoScale) the
// pending scale is not applied (a later kernel of the same step). Applies the
// pending scale on load otherwise. Block (32, BY); one thread per grid point.
// ---------------------------------------------------------------------------
// The pointwise substeps at grid point (ix, iy) of the state A (one grid),
// written to B; scale: the pending renormalisation scale per component; Ot the
// Rabi coupling Omega/sqrt2 of this step.
// Pending renormalisation scale of component j in the arithmetic type R.
template <typename R> __device__ __forceinline__ R scale_of(const DevScalars* sc, int j);
template <> __device__ __forceinline__ double scale_of<double>(const DevScalars* sc, int j) { return sc->scale[j]; }
template <> __device__ __forceinline__ float scale_of<float>(const DevScalars* sc, int j) { return sc->scale_f[j]; }
template <> __device__ __forceinline__ df scale_of<df>(const DevScalars* sc, int j) {
    return df(sc->scale_f[j], sc->scale_l[j]);
}

constexpr int kMaskReverse = 8;
constexpr int kMaskNoScale = 16;

// The state at one grid point as loaded: the three values and their raw
// differences psi(x+1) - psi(x-1), psi(y+1) - psi(y-1) (zero ghosts), before
// the pending scale is applied. Loading needs no scale, so a kernel can issue
// these loads while it still works out the scale.
template <typename R> struct PointIn {
    cx<R> u[3], X[3], Y[3];
};

template <typename R>
__device__ __forceinline__ void pointwise_load(const typename V2<R>::T* __restrict__ A, const KParams& p, int ix,
                                               int iy, bool so, PointIn<R>& in) {
    const size_t plane = (size_t)p.nx * p.ny;
    const size_t c = (size_t)iy * p.nx + ix;
    const cx<R> zero = {R(0), R(0)};
#pragma unroll
    for (int j = 0; j < 3; j++) {
        in.u[j] = ld<R>(A, j * plane + c);
        in.X[j] = zero;
        in.Y[j] = zero;
    }
    if (so) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<R> xp = (ix + 1 < p.nx) ? ld<R>(A, j * plane + c + 1) : zero;
            cx<R> xm = (ix > 0) ? ld<R>(A, j * plane + c - 1) : zero;
            in.X[j] = sub(xp, xm);
            if (p.dim == 2) {
                cx<R> yp = (iy + 1 < p.ny) ? ld<R>(A, j * plane + c + p.nx) : zero;
                cx<R> ym = (iy > 0) ? ld<R>(A, j * plane + c - p.nx) : zero;
                in.Y[j] = sub(yp, ym);
            }
        }
    }
}

// The pointwise substeps at one loaded grid point; u: the three updated values.
// ds: the pending scale per component (3 values); mask as for pointwise_point.
// STD: the full step of a 2D grid (mask 7, SO case 4) known at compile time.
template <typename R, bool IMAG, bool STD = false>
__device__ __forceinline__ void pointwise_apply(const PointIn<R>& in, const KParams& p, const R* ds, R Ot, int ix,
                                                int iy, int mask_rt, cx<R> (&u)[3]) {
    const int mask = STD ? 7 : mask_rt;
    const int so_case = STD ? 4 : p.so_case;
    const int dim = STD ? 2 : p.dim;
    R d[3];
#pragma unroll
    for (int j = 0; j < 3; j++) d[j] = ds[j];
#pragma unroll
    for (int j = 0; j < 3; j++) u[j] = scl(d[j], in.u[j]);
    const R dt = kc<R>(p, KC_DT);
    if ((mask & 1) && so_case) {
        R gx[3], gy[3];
        if (p.renorm != 2) {
            // one scale for all components (DJ2, or none): the same products, formed once
            const R g = kc<R>(p, KC_HX) * d[0], h = kc<R>(p, KC_HY) * d[0];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                gx[j] = g;
                gy[j] = h;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                gx[j] = kc<R>(p, KC_HX) * d[j];
                gy[j] = kc<R>(p, KC_HY) * d[j];
            }
        }
        so_point<IMAG>(u, in.X, in.Y, gx, gy, so_case);
    }
    auto calcnu = [&]() {
        // V = wx^2 x^2/2 + wy^2 y^2/2 with x = kx dx: kx^2 is an exact integer
        const int kx = ix - p.nx / 2, ky = iy - p.ny / 2;
        if constexpr (is_pair<R>()) {
            // the pair's points are (ix, ix + 1)
            const int kx1 = kx + 1;
            R V = kc<R>(p, KC_VX) * R((float)(kx * kx), (float)(kx1 * kx1)) +
                  (dim == 2 ? kc<R>(p, KC_VY) * R((float)(ky * ky)) : R(0));
            calcnu_point<IMAG>(u, V, kc<R>(p, KC_C0), kc<R>(p, KC_C2), dt);
        } else if constexpr (!is_f32<R>()) {
            // complex128 / double-float: -dt folded into the coefficients (exponent -dt mu directly)
            R Vn = kc<R>(p, KC_NVX) * R(kx * kx) + (dim == 2 ? kc<R>(p, KC_NVY) * R(ky * ky) : R(0));
            calcnu_point_dt<IMAG>(u, Vn, p);
        } else {
            R V = kc<R>(p, KC_VX) * R(kx * kx) + (dim == 2 ? kc<R>(p, KC_VY) * R(ky * ky) : R(0));
            calcnu_point<IMAG>(u, V, kc<R>(p, KC_C0), kc<R>(p, KC_C2), dt);
        }
    };
    auto herm = [&]() {
        if constexpr (std::is_same<R, df>::value)
            herm_point_df<IMAG>(u, kc<R>(p, KC_C2), Ot, p);
        else
            herm_point<IMAG>(u, kc<R>(p, KC_C2), Ot, dt, &p);
    };
    if (mask & kMaskReverse) {
        if (mask & 4) herm();
        if (mask & 2) calcnu();
    } else {
        if (mask & 2) calcnu();
        if (mask & 4) herm();
    }
}

// pointwise_point: load and apply at one grid point; pointwise_at stores the
// result. ds: the pending scale per component (3 values).
template <typename R, bool IMAG>
__device__ __forceinline__ void pointwise_point(const typename V2<R>::T* __restrict__ A, const KParams& p,
                                                const R* ds, R Ot, int ix, int iy, int mask, cx<R> (&u)[3]) {
    PointIn<R> in;
    pointwise_load<R>(A, p, ix, iy, (mask & 1) && p.so_case, in);
    pointwise_apply<R, IMAG>(in, p, ds, Ot, ix, iy, mask, u);
}

template <typename R, bool IMAG>
__device__ __forceinline__ void pointwise_at(const typename V2<R>::T* __restrict__ A,
                                             typename V2<R>::T* __restrict__ B, const KParams& p,
                                             const DevScalars* sc, R Ot, int ix, int iy, int mask) {
    const size_t plane = (size_t)p.nx * p.ny;
    const size_t c = (size_t)iy * p.nx + ix;
    const bool ns = (mask & kMaskNoScale) != 0;
    const R ds[3] = {ns ? R(1) : scale_of<R>(sc, 0), ns ? R(1) : scale_of<R>(sc, 1), ns ? R(1) : scale_of<R>(sc, 2)};
    cx<R> u[3];
    pointwise_point<R, IMAG>(A, p, ds, Ot, ix, iy, mask, u);
#pragma unroll
    for (int j = 0; j < 3; j++) st<R>(B, j * plane + c, u[j]);
}

template <typename R, bool IMAG>
__global__ void __launch_bounds__(128) k_pointwise(const typename V2<R>::T* __restrict__ A,
                                                   typename V2<R>::T* __restrict__ B, KParams p,
                                                   const DevScalars* __restrict__ sc,
                                                   const double* __restrict__ omega_tab, int mask) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    pdl_wait();
    if (ix >= p.nx || iy >= p.ny) return;
    const R Ot = omega_tab ? to_r<R>(__ldg(omega_tab + sc->step_idx) * 0.70710678118654752440)
                           : kc<R>(p, KC_OMEGA);
    pointwise_at<R, IMAG>(A, B, p, sc, Ot, ix, iy, mask);
}

// The same substeps for the complex64 state, two neighbouring points (ix, ix + 1)
// a thread (nx even): the three values of both points and their y neighbours
// come in 16-byte loads, the x neighbours from the pair itself and one 8-byte
// load on each side, the results go out in 16-byte stores; the arithmetic per
// point is pointwise_apply's, as in k_pointwise. The complex64 pointwise kernel
// is bound by instruction issue, half of it loads and their index arithmetic.
// The pointwise substeps of the two neighbouring points (ix, ix + 1) of row iy
// (complex64, nx even) as one f32x2 pair (lane 0: ix, lane 1: ix + 1): the
// 16-byte loads of each component's pair, the x and y neighbours (zero ghosts;
// inner points without the selects), then pointwise_apply.
template <bool IMAG, bool STD>
__device__ __forceinline__ void pair_substeps(const float2* __restrict__ A, const KParams& p, const f32x2 (&ds)[3],
                                              float Ot, int mask, int ix, int iy, cx<f32x2> (&u)[3]) {
    const size_t plane = (size_t)p.nx * p.ny;
    const size_t c = (size_t)iy * p.nx + ix;
    const bool so = STD || ((mask & 1) && p.so_case);
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float2 z2 = make_float2(0.0f, 0.0f);
    PointIn<f32x2> in;
    float4 v[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        v[j] = __ldg(reinterpret_cast<const float4*>(A + j * plane + c));
        in.u[j] = {f32x2(v[j].x, v[j].z), f32x2(v[j].y, v[j].w)};
        in.X[j] = in.Y[j] = {f32x2(0.0f), f32x2(0.0f)};
    }
    if (so) {
        // X = psi(x + 1) - psi(x - 1), Y = psi(y + 1) - psi(y - 1), zero ghosts
        auto diffs = [&](int j, float2 xm, float2 xp, float4 ym, float4 yp) {
            in.X[j] = {f32x2(v[j].z, xp.x) - f32x2(xm.x, v[j].x), f32x2(v[j].w, xp.y) - f32x2(xm.y, v[j].y)};
            in.Y[j] = {f32x2(yp.x, yp.z) - f32x2(ym.x, ym.z), f32x2(yp.y, yp.w) - f32x2(ym.y, ym.w)};
        };
        // every neighbour inside the grid (2D): loads without the zero ghosts
        const bool inner = (STD || p.dim == 2) && ix > 0 && ix + 2 < p.nx && iy > 0 && iy + 1 < p.ny;
        if (inner) {
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const float2* a = A + j * plane + c;
                diffs(j, __ldg(a - 1), __ldg(a + 2), __ldg(reinterpret_cast<const float4*>(a - p.nx)),
                      __ldg(reinterpret_cast<const float4*>(a + p.nx)));
            }
        } else {
            const bool two = STD || p.dim == 2;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const float2* a = A + j * plane + c;
                const float2 xm = ix > 0 ? __ldg(a - 1) : z2;
                const float2 xp = ix + 2 < p.nx ? __ldg(a + 2) : z2;
                const float4 ym = two && iy > 0 ? __ldg(reinterpret_cast<const float4*>(a - p.nx)) : z4;
                const float4 yp = two && iy + 1 < p.ny ? __ldg(reinterpret_cast<const float4*>(a + p.nx)) : z4;
                diffs(j, xm, xp, ym, yp);
            }
        }
    }
    pointwise_apply<f32x2, IMAG, STD>(in, p, ds, f32x2(Ot), ix, iy, mask, u);
}

// The pending scale (complex64 copy) and the Rabi coupling of this step for the pair kernels.
__device__ __forceinline__ void pair_constants(const KParams& p, const DevScalars* sc, const double* omega_tab, int mask,
                                               f32x2 (&ds)[3], float& Ot) {
    Ot = kc<float>(p, KC_OMEGA);
    if (omega_tab) Ot = to_r<float>(__ldg(omega_tab + sc->step_idx) * 0.70710678118654752440);
    const bool ns = (mask & kMaskNoScale) != 0;
#pragma unroll
    for (int j = 0; j < 3; j++) ds[j] = f32x2(ns ? 1.0f : scale_of<float>(sc, j));
}

template <bool IMAG, bool STD>
__global__ void __launch_bounds__(256) k_pointwise2(const float2* __restrict__ A, float2* __restrict__ B, KParams p,
                                                    const DevScalars* __restrict__ sc,
                                                    const double* __restrict__ omega_tab, int mask) {
    const int ix = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    pdl_wait();
    if (ix >= p.nx || iy >= p.ny) return;
    f32x2 ds[3];
    float Ot;
    pair_constants(p, sc, omega_tab, mask, ds, Ot);
    cx<f32x2> u[3];
    pair_substeps<IMAG, STD>(A, p, ds, Ot, mask, ix, iy, u);
    pdl_trigger();  // the next kernel's blocks may take the slots this grid frees
    const size_t plane = (size_t)p.nx * p.ny;
    const size_t c = (size_t)iy * p.nx + ix;
#pragma unroll
    for (int j = 0; j < 3; j++)
        *reinterpret_cast<float4*>(B + j * plane + c) = make_float4(u[j].re.v.x, u[j].im.v.x, u[j].re.v.y, u[j].im.v.y);
}

// ---------------------------------------------------------------------------
// End of a step: one block of 3 warps; warp j sums the m partial norms of
// component j (partials[j*m .. j*m + m), fixed order), then thread 0 publishes
// N_j, the next pending scale (Eq. (DJ2) / (DJ) for renorm != 0, else 1) and
// advances the step counter. Few threads on purpose: the FP64 adds run on one
// SM's FP64 pipe.
// ---------------------------------------------------------------------------
// Sum of the m partials q[0..m) by the calling warp in a fixed order (lane-
// strided into four accumulators, then a shuffle tree): the same value in every
// lane and in every block that calls it.
__device__ __forceinline__ double sum_partials_warp(const double* q, int m) {
    const int lane = threadIdx.x & 31;
    // up to 256 partials: all eight loads of a lane in flight at once, then a tree
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = (lane + 32 * k < m) ? __ldcg(q + lane + 32 * k) : 0.0;
    double s = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    for (int b = lane + 256; b < m; b += 32) s += __ldcg(q + b);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

// The same for partials held as double-float pairs (the complex64 and
// double-float forms: their sweeps sum the norms on the FP32 pipe); the tree is
// pairwise, so the sum keeps about 2^-48 * log2(m) relative accuracy.
__device__ __forceinline__ df df_shfl_xor(df v, int off) {
    return df(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}
__device__ __forceinline__ df sum_partials_warp(const df* q, int m) {
    const int lane = threadIdx.x & 31;
    const float2* q2 = reinterpret_cast<const float2*>(q);
    df v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const float2 e = (lane + 32 * k < m) ? __ldcg(q2 + lane + 32 * k) : make_float2(0.0f, 0.0f);
        v[k] = df(e.x, e.y);
    }
    df s = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    for (int b = lane + 256; b < m; b += 32) {
        const float2 e = __ldcg(q2 + b);
        s = s + df(e.x, e.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = s + df_shfl_xor(s, off);
    return s;
}

// The pending scale from double-float norm sums S_j (before the cell factor):
// Eq. (DJ2) in pairs (FP32 estimate of 1/sqrt, Newton steps; no FP64 on this
// path); Eq. (DJ) and a missing renormalisation through renorm_factors in FP64.
// f: the factor of every component as a pair (DJ2); d: the FP64 factors; N: the norms.
__device__ __forceinline__ void scale_from_df_sums(const df (&S)[3], double cell, int renorm, double mag, df (&f)[3],
                                                   double (&d)[3], double (&N)[3], bool& finite) {
    const df c = df_from(cell);
    df Nd[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        Nd[j] = S[j] * c;
        N[j] = df_to(Nd[j]);
    }
    finite = isfinite(Nd[0].hi) && isfinite(Nd[1].hi) && isfinite(Nd[2].hi);
    if (finite && renorm == 1) {
        const df Nt = (Nd[0] + Nd[1]) + Nd[2];
        const df g = Nt.hi > 0.0f ? df_rsqrt(Nt) : df(1.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            f[j] = g;
            d[j] = df_to(g);
        }
        return;
    }
    renorm_factors(N, finite ? renorm : 0, mag, d);
#pragma unroll
    for (int j = 0; j < 3; j++) f[j] = df_from(d[j]);
}

// Thread 0: N_j, the next pending scale and the step counter from the three
// component sums (FP64 sums, or double-float pairs when part_df).
__device__ __forceinline__ void finalize_publish(const double (&red)[3], const df (&red_df)[3], double cell,
                                                 int renorm, double mag, int advance_step, DevScalars* sc,
                                                 int part_df) {
    double N[3], d[3];
    bool finite;
    if (part_df) {
        const df S[3] = {red_df[0], red_df[1], red_df[2]};
        df f[3];
        scale_from_df_sums(S, cell, renorm, mag, f, d, N, finite);
    } else {
        N[0] = red[0] * cell;
        N[1] = red[1] * cell;
        N[2] = red[2] * cell;
        finite = isfinite(N[0]) && isfinite(N[1]) && isfinite(N[2]);
        renorm_factors(N, finite ? renorm : 0, mag, d);
    }
    for (int q3 = 0; q3 < 3; q3++) {
        sc->norms[q3] = N[q3];
        sc->scale[q3] = d[q3];
        sc->scale_f[q3] = (float)d[q3];
        sc->scale_l[q3] = (float)(d[q3] - (double)sc->scale_f[q3]);
    }
    if (!finite) sc->err |= 1;
    if (advance_step) sc->step_idx += 1;
    sc->scale_src = 0;
}

// part_df: the partials are double-float pairs (see sum_partials_warp above).
static __global__ void __launch_bounds__(96) k_finalize(const double* partials, int m, double cell, int renorm,
                                                 double mag, int advance_step, DevScalars* sc, int part_df) {
    __shared__ double red[3];
    __shared__ df red_df[3];
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    pdl_trigger();  // one small block: the next step's first kernel may launch now
    pdl_wait();
    if (part_df) {
        const df s = sum_partials_warp(reinterpret_cast<const df*>(partials) + (size_t)j * m, m);
        if (lane == 0) red_df[j] = s;
    } else {
        const double s = sum_partials_warp(partials + (size_t)j * m, m);
        if (lane == 0) red[j] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[3] = {red[0], red[1], red[2]};
        df rd[3] = {red_df[0], red_df[1], red_df[2]};
        finalize_publish(r, rd, cell, renorm, mag, advance_step, sc, part_df);
    }
}

// The same for more than 256 partials per component (the row-tiled sweeps of
// large grids): kFinWarps warps per component, warp s summing the partials
// s * 32 + lane + 256 k in batches of eight loads in flight (a pairwise tree
// per batch, the batches in order), then the warps' sums in index order. The
// order depends on m only: the same sums on every run.
constexpr int kFinWarps = 8;
template <typename P> __device__ __forceinline__ P fin_load(const P* q, int i, int m);
template <> __device__ __forceinline__ double fin_load<double>(const double* q, int i, int m) {
    return i < m ? __ldcg(q + i) : 0.0;
}
template <> __device__ __forceinline__ df fin_load<df>(const df* q, int i, int m) {
    if (i >= m) return df(0.0f, 0.0f);
    const float2 e = __ldcg(reinterpret_cast<const float2*>(q) + i);
    return df(e.x, e.y);
}
__device__ __forceinline__ double fin_xor(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ df fin_xor(df v, int off) { return df_shfl_xor(v, off); }

template <typename P> __device__ __forceinline__ P sum_partials_wide(const P* q, int m, int sub) {
    const int lane = threadIdx.x & 31;
    P s = P(0);
    for (int b0 = sub * 32 + lane; b0 < m; b0 += 8 * 32 * kFinWarps) {
        P v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = fin_load(q, b0 + k * 32 * kFinWarps, m);
        s = s + (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = s + fin_xor(s, off);
    return s;
}

static __global__ void __launch_bounds__(96 * kFinWarps) k_finalize_wide(const double* partials, int m, double cell,
                                                                      int renorm, double mag, int advance_step,
                                                                      DevScalars* sc, int part_df) {
    __shared__ double red[3][kFinWarps];
    __shared__ df red_df[3][kFinWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = warp / kFinWarps, sub = warp % kFinWarps;
    // the y sweep lets this block become resident early; the next step's first
    // kernel launches once the sweep is done
    pdl_wait();
    pdl_trigger();
    if (part_df) {
        const df s = sum_partials_wide(reinterpret_cast<const df*>(partials) + (size_t)j * m, m, sub);
        if (lane == 0) red_df[j][sub] = s;
    } else {
        const double s = sum_partials_wide(partials + (size_t)j * m, m, sub);
        if (lane == 0) red[j][sub] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[3];
        df rd[3];
        for (int c = 0; c < 3; c++) {
            r[c] = red[c][0];
            rd[c] = red_df[c][0];
            for (int w = 1; w < kFinWarps; w++) {
                r[c] += red[c][w];
                rd[c] = rd[c] + red_df[c][w];
            }
        }
        finalize_publish(r, rd, cell, renorm, mag, advance_step, sc, part_df);
    }
}

// ---------------------------------------------------------------------------
// COEF: build the Crank-Nicolson tables of one axis for bt = (bre, bim)
// (bt = dt/(4h^2) in imaginary time, i dt/(4h^2) in real time). One thread;
// FP64 arithmetic, stored rounded to R.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double* r, double* i) {
    // (a / b) with Smith's scaling
    if (fabs(br) >= fabs(bi)) {
        double q = bi / br, den = br + bi * q;
        *r = (ar + ai * q) / den;
        *i = (ai - ar * q) / den;
    } else {
        double q = br / bi, den = bi + br * q;
        *r = (ar * q + ai) / den;
        *i = (ai * q - ar) / den;
    }
}

// Tables have len entries (a multiple of the chunk length C); entries past n
// are zero (fa = fg = 0, hence the chunk products vanish there too). With
// interleave (lines longer than 1024 points) entry i of every table is stored at
// (i % C) * (len / C) + i / C: lane g of a line's warp group reads its chunk
// entry m at m * G + g, G = len / C lanes, so a warp's table reads are coalesced.
template <typename R>
__global__ void k_coef(typename V2<R>::T* fa, typename V2<R>::T* fg, typename V2<R>::T* fp,
                       typename V2<R>::T* fq, int n, int C, int len, int interleave, double bre, double bim) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double dr = 1.0 + 2.0 * bre, di = 2.0 * bim;  // diagonal 1 + 2 bt
    const cx<R> zero = {R(0), R(0)};
    const int G = len / C;
    auto at = [&](int i) { return interleave ? (i % C) * G + i / C : i; };
    for (int i = n; i < len; i++) {
        st<R>(fa, at(i), zero);
        st<R>(fg, at(i), zero);
    }
    double ur = dr, ui = di;
    for (int i = 0; i < n; i++) {
        if (i > 0) {
            // u_i = (1 + 2bt) - bt^2 / u_{i-1}
            double b2r = bre * bre - bim * bim, b2i = 2.0 * bre * bim;
            double qr, qi;
            cdiv(b2r, b2i, ur, ui, &qr, &qi);
            ur = dr - qr;
            ui = di - qi;
        }
        double ar, ai, gr, gi;
        cdiv(1.0, 0.0, ur, ui, &ar, &ai);
        cdiv(bre, bim, ur, ui, &gr, &gi);
        st<R>(fa, at(i), cx<R>{to_r<R>(ar), to_r<R>(ai)});
        st<R>(fg, at(i), cx<R>{to_r<R>(gr), to_r<R>(gi)});
    }
    // chunk products, computed from the rounded-to-FP64 fg values
    for (int k0 = 0; k0 < len; k0 += C) {
        int k1 = k0 + C;
        double Pr = 1.0, Pi = 0.0;
        for (int i = k0; i < k1; i++) {
            const cx<R> g = unpack(fg[at(i)]);
            double gr = dbl(g.re), gi = dbl(g.im);
            double tr = Pr * gr - Pi * gi, ti = Pr * gi + Pi * gr;
            Pr = tr;
            Pi = ti;
            st<R>(fp, at(i), cx<R>{to_r<R>(Pr), to_r<R>(Pi)});
        }
        Pr = 1.0;
        Pi = 0.0;
        for (int i = k1 - 1; i >= k0; i--) {
            const cx<R> g = unpack(fg[at(i)]);
            double gr = dbl(g.re), gi = dbl(g.im);
            double tr = Pr * gr - Pi * gi, ti = Pr * gi + Pi * gr;
            Pr = tr;
            Pi = ti;
            st<R>(fq, at(i), cx<R>{to_r<R>(Pr), to_r<R>(Pi)});
        }
    }
}

// ---------------------------------------------------------------------------
// Apply the pending scale in place (psi_j <- d_j psi_j).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_flush(typename V2<R>::T* A, size_t plane, const DevScalars* sc) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = 3 * plane;
    for (; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(i / plane);
        R d = to_r<R>(sc->scale[j]);
        cx<R> v = ldc<R>(A, i);
        st<R>(A, i, scl(d, v));
    }
}

static __global__ void k_reset_scale(DevScalars* sc) {
    if (threadIdx.x < 4) {
        sc->scale[threadIdx.x] = 1.0;
        sc->scale_f[threadIdx.x] = 1.0f;
        sc->scale_l[threadIdx.x] = 0.0f;
    }
    if (threadIdx.x == 0) sc->scale_src = 0;
}

// ---------------------------------------------------------------------------
// Norms of the state (no pending scale): per-block FP64 partials, last block
// publishes N_j and, for renorm != 0, the renormalisation scale.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_norms(const typename V2<R>::T* A, size_t plane, double cell, int renorm,
                                               double mag, double* partials, DevScalars* sc, int advance) {
    __shared__ double red[8 * 3];
    double v[3] = {0.0, 0.0, 0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * plane;
         i += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(i / plane);
        cx<R> a = ldc<R>(A, i);
        double q = dbl(a.re) * dbl(a.re) + dbl(a.im) * dbl(a.im);
        if (j == 0) v[0] += q;
        else if (j == 1) v[1] += q;
        else v[2] += q;
    }
    block_reduce<3>(v, red);
    if (threadIdx.x == 0)
        for (int j = 0; j < 3; j++) partials[3 * blockIdx.x + j] = v[j];
    if (last_block(&sc->ticket[2]))
        finalize_norms(partials, gridDim.x, cell, renorm, mag, advance != 0, sc, &sc->ticket[2]);
}

// ---------------------------------------------------------------------------
// Observables (Eq. (noma), Eq. (energy), rms sizes) of the state (no pending
// scale). Per point in FP64: N_j, r^2 rho_j, the kinetic energy of the links
// ending at the point (plus the ghost links at the upper edges), trap,
// interaction, Rabi and SO energy densities.
// ---------------------------------------------------------------------------
constexpr int NACC = 11;

// The FP64 observable densities of grid point (ix, iy) of one grid, added to v.
template <typename R>
__device__ __forceinline__ void obs_point(const typename V2<R>::T* __restrict__ A, const KParams& p, double omega_t,
                                          int ix, int iy, double (&v)[NACC]) {
    {
        const size_t plane = (size_t)p.nx * p.ny;
        const size_t c = (size_t)iy * p.nx + ix;
        cx<double> u[3];
        const cx<double> zero = {0.0, 0.0};
        for (int j = 0; j < 3; j++) {
            cx<R> a = ld<R>(A, j * plane + c);
            u[j] = {dbl(a.re), dbl(a.im)};
        }
        double x = (ix - p.nx / 2) * p.dx, y = (p.dim == 2) ? (iy - p.ny / 2) * p.dy : 0.0;
        double rr = x * x + y * y;
        double rp = nrm(u[0]), r0 = nrm(u[1]), rm = nrm(u[2]), rho = rp + r0 + rm;
        v[0] = rp;
        v[1] = r0;
        v[2] = rm;
        v[3] = rr * rp;
        v[4] = rr * r0;
        v[5] = rr * rm;
        // kinetic: links (ix-1, ix) and, at the upper edge, (ix, ghost); same in y
        double ek = 0.0;
        const double idx2 = 1.0 / (p.dx * p.dx), idy2 = 1.0 / (p.dy * p.dy);
        cx<double> X[3], Y[3];
        for (int j = 0; j < 3; j++) {
            cx<double> xm = zero, xp = zero, ym = zero, yp = zero;
            if (ix > 0) {
                cx<R> a = ld<R>(A, j * plane + c - 1);
                xm = {dbl(a.re), dbl(a.im)};
            }
            if (ix + 1 < p.nx) {
                cx<R> a = ld<R>(A, j * plane + c + 1);
                xp = {dbl(a.re), dbl(a.im)};
            }
            ek += 0.5 * nrm(sub(u[j], xm)) * idx2;
            if (ix == p.nx - 1) ek += 0.5 * nrm(u[j]) * idx2;
            X[j] = sub(xp, xm);
            if (p.dim == 2) {
                if (iy > 0) {
                    cx<R> a = ld<R>(A, j * plane + c - p.nx);
                    ym = {dbl(a.re), dbl(a.im)};
                }
                if (iy + 1 < p.ny) {
                    cx<R> a = ld<R>(A, j * plane + c + p.nx);
                    yp = {dbl(a.re), dbl(a.im)};
                }
                ek += 0.5 * nrm(sub(u[j], ym)) * idy2;
                if (iy == p.ny - 1) ek += 0.5 * nrm(u[j]) * idy2;
                Y[j] = sub(yp, ym);
            } else {
                Y[j] = zero;
            }
        }
        v[6] = ek;
        double V = p.wx2h * x * x + (p.dim == 2 ? p.wy2h * y * y : 0.0);
        v[7] = V * rho;
        cx<double> X4 = mul(cmul(u[2], mul(u[1], u[1])), cj(u[0]));  // psi_-^* psi_0^2 psi_+^*
        v[8] = 0.5 * (p.c0 * rho * rho +
                      p.c2 * (rp * rp + rm * rm + 2.0 * rp * r0 + 2.0 * rm * r0 - 2.0 * rp * rm + 4.0 * X4.re));
        cx<double> Rb = cmul(add(u[0], u[2]), u[1]);  // (psi_+^* + psi_-^*) psi_0
        v[9] = 2.0 * omega_t * Rb.re;
        if (p.so_case) {
            // H_SO psi via the SO update with unit time factor on a zero state
            cx<double> h[3] = {zero, zero, zero};
            double gx[3] = {p.sx, p.sx, p.sx}, gy[3] = {p.sy, p.sy, p.sy};
            so_point<true>(h, X, Y, gx, gy, p.so_case);  // h = -(H_SO psi)
            v[10] = -(cmul(u[0], h[0]).re + cmul(u[1], h[1]).re + cmul(u[2], h[2]).re);
        }
    }
}

// The SGPE_NOBS observables from the grid sums s (obs_point summed over the grid).
__device__ __forceinline__ void obs_finish(const double (&s)[NACC], double w, double* o, int* err) {
    double N0 = s[0] * w, N1 = s[1] * w, N2 = s[2] * w, Nt = N0 + N1 + N2;
    double ekin = s[6] * w, etrap = s[7] * w, eint = s[8] * w, erabi = s[9] * w, eso = s[10] * w;
    o[0] = N0;
    o[1] = N1;
    o[2] = N2;
    o[3] = Nt;
    o[4] = N0 - N2;
    o[5] = ekin + etrap + eint + erabi + eso;
    o[6] = Nt > 0.0 ? (ekin + etrap + eso + erabi + 2.0 * eint) / Nt : 0.0;
    o[7] = s[0] > 0.0 ? sqrt(s[3] / s[0]) : 0.0;
    o[8] = s[1] > 0.0 ? sqrt(s[4] / s[1]) : 0.0;
    o[9] = s[2] > 0.0 ? sqrt(s[5] / s[2]) : 0.0;
    double ss = s[0] + s[1] + s[2];
    o[10] = ss > 0.0 ? sqrt((s[3] + s[4] + s[5]) / ss) : 0.0;
    o[11] = ekin;
    o[12] = etrap;
    o[13] = eint;
    o[14] = erabi;
    o[15] = eso;
    if (!(isfinite(Nt))) *err |= 1;
}

template <typename R>
__global__ void __launch_bounds__(128) k_observables(const typename V2<R>::T* __restrict__ A, KParams p, double omega_t,
                                                     double* partials, DevScalars* sc) {
    __shared__ double red[4 * NACC];
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y * blockDim.y + threadIdx.y;
    double v[NACC];
#pragma unroll
    for (int q = 0; q < NACC; q++) v[q] = 0.0;
    if (ix < p.nx && iy < p.ny) obs_point<R>(A, p, omega_t, ix, iy, v);
    // block reduce (blockDim.x * blockDim.y threads, flattened)
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int q = 0; q < NACC; q++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    if (lane == 0)
        for (int q = 0; q < NACC; q++) red[warp * NACC + q] = v[q];
    __syncthreads();
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    if (tid == 0) {
        for (int q = 0; q < NACC; q++) {
            double s = 0.0;
            for (int w = 0; w < nw; w++) s += red[w * NACC + q];
            partials[(size_t)blk * NACC + q] = s;
        }
    }
    __shared__ bool am_last;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned t = atomicAdd(&sc->ticket[1], 1u);
        am_last = (t == gridDim.x * gridDim.y - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const int nblk = gridDim.x * gridDim.y;
    if (tid < 32) {
        double s[NACC];
        for (int q = 0; q < NACC; q++) s[q] = 0.0;
        for (int b = tid; b < nblk; b += 32)
            for (int q = 0; q < NACC; q++) s[q] += __ldcg(partials + (size_t)b * NACC + q);
        for (int q = 0; q < NACC; q++)
            for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
        if (tid == 0) {
            obs_finish(s, p.cell, sc->obs, &sc->err);
            sc->ticket[1] = 0u;
        }
    }
}

}  // namespace sgpe
