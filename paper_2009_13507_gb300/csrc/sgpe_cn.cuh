// sgpe_cn.cuh -- Crank-Nicolson sweeps (Sec. 3, LU / LUX / LUY) with each
// lane's chunk of a line held in registers; compile-time chunk length C.
//
// A line of n points is split into 32 chunks of C = next_pow2(ceil(n/32))
// points (n <= 1024); lane l owns points [lC, lC + C). The coefficient tables
// are padded to 32*C entries with zeros beyond n, and points beyond n load as
// zero, so a ragged line needs no special case: the recurrences stay at zero
// past the end and the chunk products there vanish.
//
// One warp per block: the FP64 sweeps are bound by the FP64 pipe of each SM,
// so the work is cut into as many equal blocks as there are lines (x) or
// column pairs (y) for an even spread over the 152 SMs.
#pragma once
#include "sgpe_kernels.cuh"

namespace sgpe {

// A lane's slice [i0, i0 + C) of one coefficient table: held in registers when
// PRE (loaded once, up front, with the other loads of the kernel) or read from
// global memory at each use.
template <typename R, int C, bool PRE> struct ChunkTab {
    cx<R> r[PRE ? C : 1];
    const typename V2<R>::T* p;
    __device__ __forceinline__ void init(const typename V2<R>::T* base, int i0) {
        p = base + i0;
        if (PRE) {
#pragma unroll
            for (int m = 0; m < C; m++) r[PRE ? m : 0] = tld<R>(p, m);
        }
    }
    __device__ __forceinline__ cx<R> operator[](int m) const { return PRE ? r[PRE ? m : 0] : tld<R>(p, m); }
};

// Register-resident tables for small chunks, except FP64 real-time tables (complex, too many registers).
template <typename R, bool IMAG, int C> struct TabPolicy {
    static constexpr bool PRE = C <= 8 && (sizeof(R) == 4 || IMAG);
};

template <typename R, bool IMAG, int C> struct LaneTabs {
    static constexpr bool PRE = TabPolicy<R, IMAG, C>::PRE;
    ChunkTab<R, C, PRE> fa, fg, fp, fq;
    __device__ __forceinline__ void init(const Tabs<R>& t, int i0) {
        fa.init(t.fa, i0);
        fg.init(t.fg, i0);
        fp.init(t.fp, i0);
        fq.init(t.fq, i0);
    }
};

// Solve T w = x for the lane's chunk v (in: x, out: w), all 32 lanes together.
// SKEW: T has opposite off-diagonals (lower -a, upper +a; the Crank-Nicolson
// matrix of a first-derivative operator): the backward recurrence then runs with
// -fg and fq holds the chunk products of -fg (k_coef_skew).
template <typename R, bool IMAG, int C, bool SKEW = false>
__device__ __forceinline__ void solve_chunk(cx<R> (&v)[C], const LaneTabs<R, IMAG, C>& t) {
    const int lane = threadIdx.x & 31;
    cx<R> y = {R(0), R(0)};
#pragma unroll
    for (int m = 0; m < C; m++) {
        y = tfma<IMAG>(t.fg[m], y, tmul<IMAG>(t.fa[m], v[m]));
        v[m] = y;
    }
    cx<R> A = t.fp[C - 1], B = y;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        cx<R> Ap = shup(A, off), Bp = shup(B, off);
        if (lane >= off) {
            B = tfma<IMAG>(A, Bp, B);
            A = tmul<IMAG>(A, Ap);
        }
        if (scan_done(lane < 2 * off, A)) break;  // see tiny_carry
    }
    cx<R> cin = shup(B, 1);
    if (lane == 0) cin = {R(0), R(0)};
    cx<R> w = {R(0), R(0)};
#pragma unroll
    for (int m = C - 1; m >= 0; m--) {
        cx<R> yi = tfma<IMAG>(t.fp[m], cin, v[m]);
        if (SKEW) {
            const cx<R> g = t.fg[m];
            w = tfma<IMAG>(cx<R>{-g.re, -g.im}, w, yi);
        } else {
            w = tfma<IMAG>(t.fg[m], w, yi);
        }
        v[m] = w;
    }
    A = t.fq[0];
    B = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        cx<R> An = shdn(A, off), Bn = shdn(B, off);
        if (lane + off < 32) {
            B = tfma<IMAG>(A, Bn, B);
            A = tmul<IMAG>(A, An);
        }
        if (scan_done(lane + 2 * off >= 32, A)) break;
    }
    cx<R> cb = shdn(B, 1);
    if (lane == 31) cb = {R(0), R(0)};
#pragma unroll
    for (int m = 0; m < C; m++) v[m] = tfma<IMAG>(t.fq[m], cb, v[m]);
}

// Increment form of the sweep, used for the complex64 state: out = x + 2 e with
// T e = bt L x, L x = (x_{i-1} - x_i) + (x_{i+1} - x_i). The FP32-rounded LU
// factors then only touch the small increment e, so the sweep stays unitary
// (real time) to far better than one ulp per step; the two differences of
// neighbouring values are exact. bt is recovered from the tables as fg_0/fa_0.
// In place on the lane's chunk v (in: x, out: bt L x); all 32 lanes.
template <typename R, bool IMAG, int C>
__device__ __forceinline__ void cn_increment_rhs(cx<R> (&v)[C], const Tabs<R>& t) {
    const int lane = threadIdx.x & 31;
    const cx<R> a0 = tld<R>(t.fa, 0), g0 = tld<R>(t.fg, 0);
    cx<R> bt;
    if (IMAG) {
        bt = {g0.re / a0.re, R(0)};
    } else {
        const R den = nrm(a0);
        const cx<R> q = cmul(a0, g0);  // conj(a0) g0
        bt = {q.re / den, q.im / den};
    }
    cx<R> prev = shup(v[C - 1], 1), last = shdn(v[0], 1);
    if (lane == 0) prev = {R(0), R(0)};
    if (lane == 31) last = {R(0), R(0)};
#pragma unroll
    for (int m = 0; m < C; m++) {
        const cx<R> cur = v[m];
        const cx<R> nxt = (m + 1 < C) ? v[m + 1] : last;
        v[m] = tmul<IMAG>(bt, add(sub(prev, cur), sub(nxt, cur)));
        prev = cur;
    }
}

// Columns per warp of the y sweep and whether a lane keeps its input chunk in
// registers (small chunks) or reloads it for the final 2w - x (large chunks).
template <typename R, int C> struct CnShape {
    // complex128: one column per warp (the FP64 sweep is latency-bound, more
    // warps per SM help more than full 32-byte rows); complex64: two columns
    static constexpr int K = (sizeof(R) == 4 && C <= 8) ? 2 : 1;
    static constexpr bool KEEP = C <= 8;
};

// Per-lane accumulator of |o|^2 over the lane's points for the FP64 norm
// partials. complex64 state: each square is split exactly into p + e
// (p = x*x, e = fma(x, x, -p)) and summed as an unevaluated FP32 pair
// (Knuth's TwoSum for the high part, the rounding errors collected in the low
// part): about 2^-44 relative, i.e. FP64-grade for the few dozen terms of a
// lane, on the FP32 pipe instead of GB300's much slower FP64 pipe.
template <typename R> struct NormAcc;
// complex128 and double-float: real and imaginary squares in two accumulators,
// which halves the dependent chain of a lane's sum.
template <> struct NormAcc<double> {
    double sr = 0.0, si = 0.0;
    __device__ __forceinline__ void add(cx<double> o) {
        sr = fma(o.re, o.re, sr);
        si = fma(o.im, o.im, si);
    }
    __device__ __forceinline__ double value() const { return sr + si; }
};
template <> struct NormAcc<df> {
    df sr = df(0), si = df(0);
    __device__ __forceinline__ void add(cx<df> o) {
        sr = fma(o.re, o.re, sr);
        si = fma(o.im, o.im, si);
    }
    __device__ __forceinline__ double value() const { return df_to(sr + si); }
};
template <> struct NormAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add1(float x) {
        const float p = x * x;
        const float e = fmaf(x, x, -p);
        const float t = hi + p;
        const float bp = t - hi;
        lo += ((hi - (t - bp)) + (p - bp)) + e;
        hi = t;
    }
    __device__ __forceinline__ void add(cx<float> o) {
        add1(o.re);
        add1(o.im);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Norm partial type of the sweeps' step-ending sums: FP64 for the complex128
// state, a double-float pair (FP32 pipe) for the complex64 and double-float forms.
template <typename R> struct PartT { using T = df; };
template <> struct PartT<double> { using T = double; };

template <typename P, typename Acc> __device__ __forceinline__ P acc_value(const Acc& a);
template <> __device__ __forceinline__ double acc_value<double, NormAcc<double>>(const NormAcc<double>& a) {
    return a.value();
}
template <> __device__ __forceinline__ double acc_value<double, NormAcc<float>>(const NormAcc<float>& a) {
    return a.value();
}
template <> __device__ __forceinline__ double acc_value<double, NormAcc<df>>(const NormAcc<df>& a) {
    return a.value();
}
template <> __device__ __forceinline__ df acc_value<df, NormAcc<float>>(const NormAcc<float>& a) {
    return fast_two_sum(a.hi, a.lo);
}
template <> __device__ __forceinline__ df acc_value<df, NormAcc<df>>(const NormAcc<df>& a) { return a.sr + a.si; }

__device__ __forceinline__ df warp_sum(df v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v = v + df(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ---------------------------------------------------------------------------
// CN along x: block = one warp = one line (line = j*ny + iy). With partials
// non-null the block writes the FP64 norm of its output line to partials[line]
// (the lines of component j are contiguous).
// ---------------------------------------------------------------------------
// One x line of n points by the calling warp: input point i (i < n) comes from
// load(i), output point i goes to out[base + i]; part (nullable): the partial
// slot of this line (FP64 norm of the output line).
template <typename R, bool IMAG, int C, typename Load>
__device__ __forceinline__ void cnx_solve_line(Load load, typename V2<R>::T* out, size_t base, int n,
                                               const Tabs<R>& t, double* part) {
    constexpr bool KEEP = CnShape<R, C>::KEEP;
    const int lane = threadIdx.x & 31;
    const int i0 = lane * C;
    const cx<R> zero = {R(0), R(0)};
    LaneTabs<R, IMAG, C> lt;
    lt.init(t, i0);
    cx<R> x[KEEP ? C : 1], v[C];
#pragma unroll
    for (int m = 0; m < C; m++) {
        v[m] = (i0 + m < n) ? load(i0 + m) : zero;
        if (KEEP) x[m] = v[m];
    }
    constexpr bool INC = sizeof(R) == 4;
    if constexpr (INC) cn_increment_rhs<R, IMAG, C>(v, t);
    solve_chunk<R, IMAG, C>(v, lt);
    // complex64: only the stores remain, let the next step kernel launch (the
    // FP64 form measured faster with the implicit trigger at completion)
    if (sizeof(R) == 4) pdl_trigger();
    NormAcc<R> acc;
#pragma unroll
    for (int m = 0; m < C; m++) {
        if (i0 + m < n) {
            cx<R> xm = KEEP ? x[m] : load(i0 + m);
            cx<R> o = INC ? cx<R>{fma(R(2), v[m].re, xm.re), fma(R(2), v[m].im, xm.im)}
                          : cx<R>{fma(R(2), v[m].re, -xm.re), fma(R(2), v[m].im, -xm.im)};
            st<R>(out, base + i0 + m, o);
            if (part) acc.add(o);
        }
    }
    if (part) {
        const double t = warp_sum(acc.value());
        if (lane == 0) *part = t;
    }
}

// One x line of one grid (line = j*ny + iy) from global memory.
template <typename R, bool IMAG, int C>
__device__ __forceinline__ void cnx_line(const typename V2<R>::T* in, typename V2<R>::T* out, const KParams& p,
                                         const Tabs<R>& t, int line, double* part) {
    const size_t base = (size_t)line * p.nx;
    cnx_solve_line<R, IMAG, C>([&](int i) { return ldc<R>(in, base + i); }, out, base, p.nx, t, part);
}

template <typename R, bool IMAG, int C>
__global__ void __launch_bounds__(32) k_cnx_reg(const typename V2<R>::T* in, typename V2<R>::T* out, KParams p,
                                                Tabs<R> t, double* partials) {
    pdl_wait();
    cnx_line<R, IMAG, C>(in, out, p, t, blockIdx.x, partials ? partials + blockIdx.x : nullptr);
}

// ---------------------------------------------------------------------------
// Fused head of a 2D step, one block per grid row iy (rows of at most 1024
// points). First the pending renormalisation scale: when the previous step's
// y sweep left its norm partials (DevScalars::scale_src), warps 0..2 sum the m
// partials of their component and thread 0 forms the scale (Eq. (DJ2) / (DJ));
// every block does the same sums in the same order, so all blocks agree and no
// separate end-of-step launch is needed. Then all threads run the pointwise
// substeps (SO, CALCNU, HERM) of the row's points for the three components and
// stage the results in shared memory in the lanes' chunk layout, each chunk
// padded to C + 1 entries so that a lane's chunk reads are free of bank
// conflicts; then warp j solves the Crank-Nicolson x line of component j from
// there and writes it to B.
// ---------------------------------------------------------------------------
constexpr int kPwxThreads = 256;

template <typename R, int C> constexpr size_t pwx_smem_bytes() {
    return (size_t)3 * 32 * (C + 1) * sizeof(typename V2<R>::T);
}

// Two blocks per SM (at most 128 registers a thread) for rows of up to 512
// points, except the complex64 real-time form at 512 points, which measured
// faster with one block and its unconstrained registers (512^2 real time:
// complex128 199 -> 179, double-float 154 -> 94, complex64 63 -> 67 us/step).
template <typename R, int C, bool IMAG> constexpr int pwx_min_blocks() {
    return (C <= 8 || (C <= 16 && !(sizeof(R) == 4 && !IMAG))) ? 2 : 1;
}

template <typename R, bool IMAG, int C>
__global__ void __launch_bounds__(kPwxThreads, pwx_min_blocks<R, C, IMAG>())
    k_pwx(const typename V2<R>::T* __restrict__ A, typename V2<R>::T* __restrict__ B, KParams p,
          const DevScalars* __restrict__ sc, const double* __restrict__ omega_tab, Tabs<R> t,
          const double* __restrict__ partials, int m, int renorm) {
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char pwx_smem[];
    T* row = reinterpret_cast<T*>(pwx_smem);
    __shared__ double red[3];
    __shared__ R ds[3];
    constexpr int S = 32 * (C + 1);  // staged entries per component
    const int iy = blockIdx.x;
    const int nx = p.nx;
    const int warp = threadIdx.x >> 5;
    pdl_wait();
    // the row's loads first (they need no scale), then the scale, then the substeps
    constexpr int PPT = (32 * C + kPwxThreads - 1) / kPwxThreads;  // points per thread
    PointIn<R> in[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int ix = threadIdx.x + k * kPwxThreads;
        if (ix < nx) pointwise_load<R>(A, p, ix, iy, p.so_case != 0, in[k]);
    }
    // Complex128: with one pending scale d for all components (renorm != 2) the SO
    // substep commutes with it: d psi - z h(d X) = d (psi - z h(X)). SO is then
    // applied to the raw values while warps 0..2 sum the norm partials (warps 3..7
    // before the first barrier, warps 0..2 while lane 0 of warp 7 forms the scale),
    // and the scale afterwards with the other substeps: the FP64 pipe, otherwise
    // idle during the sums, takes the SO work (256^2: 43.7 -> 42.7 us/step). The
    // FP32-pipe forms keep SO after the scale (double-float measured 19.4 -> 21.0).
    constexpr bool kSoEarly = std::is_same<R, double>::value;
    const bool so_early = kSoEarly && p.so_case != 0 && p.renorm != 2;
    auto so_raw = [&]() {
        if (!so_early) return;
        const R g = kc<R>(p, KC_HX), h = kc<R>(p, KC_HY);
        const R gx[3] = {g, g, g}, gy[3] = {h, h, h};
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int ix = threadIdx.x + k * kPwxThreads;
            if (ix < nx) so_point<IMAG>(in[k].u, in[k].X, in[k].Y, gx, gy, p.so_case);
        }
    };
    constexpr int kScaleThread = kSoEarly ? kPwxThreads - 32 : 0;  // lane 0 of the last warp (complex128)
    if (*(volatile const int*)&sc->scale_src && !std::is_same<R, double>::value) {
        // complex64 / double-float: the y sweep left double-float partials
        __shared__ df red_df[3];
        if (warp < 3) {
            const df s = sum_partials_warp(reinterpret_cast<const df*>(partials) + (size_t)warp * m, m);
            if ((threadIdx.x & 31) == 0) red_df[warp] = s;
        } else {
            so_raw();
        }
        __syncthreads();
        if (threadIdx.x == kScaleThread) {
            const df S[3] = {red_df[0], red_df[1], red_df[2]};
            df f[3];
            double d[3], N[3];
            bool finite;
            scale_from_df_sums(S, p.cell, renorm, p.mag, f, d, N, finite);
#pragma unroll
            for (int j = 0; j < 3; j++) ds[j] = to_r_df<R>(f[j]);
        }
        if (warp < 3) so_raw();
    } else if (*(volatile const int*)&sc->scale_src) {
        if (warp < 3) {
            const double s = sum_partials_warp(partials + (size_t)warp * m, m);
            if ((threadIdx.x & 31) == 0) red[warp] = s;
        } else {
            so_raw();
        }
        __syncthreads();
        if (threadIdx.x == kScaleThread) {
            double N[3] = {red[0] * p.cell, red[1] * p.cell, red[2] * p.cell};
            const bool finite = isfinite(N[0]) && isfinite(N[1]) && isfinite(N[2]);
            double d[3];
            renorm_factors(N, finite ? renorm : 0, p.mag, d);
#pragma unroll
            for (int j = 0; j < 3; j++) ds[j] = to_r<R>(d[j]);
        }
        if (warp < 3) so_raw();
    } else {
        if (threadIdx.x < 3) ds[threadIdx.x] = scale_of<R>(sc, threadIdx.x);
        so_raw();
    }
    __syncthreads();
    const R Ot = omega_tab ? to_r<R>(__ldg(omega_tab + sc->step_idx) * 0.70710678118654752440)
                           : kc<R>(p, KC_OMEGA);
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int ix = threadIdx.x + k * kPwxThreads;
        if (ix < nx) {
            cx<R> u[3];
            pointwise_apply<R, IMAG>(in[k], p, ds, Ot, ix, iy, so_early ? 6 : 7, u);
            const int slot = (ix / C) * (C + 1) + (ix % C);
#pragma unroll
            for (int j = 0; j < 3; j++) row[j * S + slot] = pack(u[j]);
        }
    }
    __syncthreads();
    if (warp < 3) {
        const T* r = row + warp * S;
        const size_t base = ((size_t)warp * p.ny + iy) * nx;
        cnx_solve_line<R, IMAG, C>([&](int i) { return unpack(r[(i / C) * (C + 1) + (i % C)]); }, B, base, nx, t,
                                   nullptr);
    }
}

// ---------------------------------------------------------------------------
// The whole 1D step loop in one block (lines of at most 1024 points): the
// three component lines live in shared memory for all nsteps steps, so a step
// costs no launch and no global traffic. Per step: the pointwise substeps of
// every point (pending scale, SO, CALCNU, HERM) into the padded chunk staging
// area, the x sweep of component j by warp j back into the state, each warp's
// FP64 norm partial, then thread 0 forms the next pending scale (Eq. (DJ2) /
// (DJ)). At the end the state goes back to A and the last norms and the
// pending scale are published, as after the multi-launch path. One SM carries
// the whole grid, which suits the complex64 and double-float forms (FP32
// pipe); the complex128 form keeps the multi-launch path, whose pointwise
// kernel spreads its FP64 work over several SMs.
// ---------------------------------------------------------------------------
constexpr int kStep1dThreads = 256;

template <typename R, int C> constexpr size_t step1d_smem_bytes(int nx) {
    return ((size_t)3 * nx + (size_t)3 * 32 * (C + 1)) * sizeof(typename V2<R>::T);
}

template <typename R, bool IMAG, int C>
__global__ void __launch_bounds__(kStep1dThreads, 1)
    k_step1d(typename V2<R>::T* __restrict__ A, KParams p, DevScalars* sc, const double* __restrict__ omega_tab,
             Tabs<R> t, int nsteps, int renorm) {
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char step1d_smem[];
    const int nx = p.nx;
    T* st_ = reinterpret_cast<T*>(step1d_smem);  // state [3][nx]
    T* stage = st_ + 3 * nx;                     // [3][32 (C + 1)]
    constexpr int S = 32 * (C + 1);
    constexpr int PPT = (32 * C + kStep1dThreads - 1) / kStep1dThreads;
    __shared__ R ds[3];
    __shared__ double red[3], dlast[3];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 3 * nx; i += kStep1dThreads) st_[i] = __ldcg(A + i);
    if (threadIdx.x < 3) {
        ds[threadIdx.x] = scale_of<R>(sc, threadIdx.x);
        dlast[threadIdx.x] = sc->scale[threadIdx.x];
    }
    const int step0 = sc->step_idx;
    const cx<R> zero = {R(0), R(0)};
    bool finite = true;
    __syncthreads();
    for (int s = 0; s < nsteps; s++) {
        const R Ot = omega_tab ? to_r<R>(__ldg(omega_tab + step0 + s) * 0.70710678118654752440) : kc<R>(p, KC_OMEGA);
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int ix = threadIdx.x + k * kStep1dThreads;
            if (ix < nx) {
                PointIn<R> in;
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    in.u[j] = unpack(st_[j * nx + ix]);
                    const cx<R> xp = ix + 1 < nx ? unpack(st_[j * nx + ix + 1]) : zero;
                    const cx<R> xm = ix > 0 ? unpack(st_[j * nx + ix - 1]) : zero;
                    in.X[j] = sub(xp, xm);
                    in.Y[j] = zero;
                }
                cx<R> u[3];
                pointwise_apply<R, IMAG>(in, p, ds, Ot, ix, 0, 7, u);
                const int slot = (ix / C) * (C + 1) + (ix % C);
#pragma unroll
                for (int j = 0; j < 3; j++) stage[j * S + slot] = pack(u[j]);
            }
        }
        __syncthreads();
        if (warp < 3) {
            const T* r = stage + warp * S;
            cnx_solve_line<R, IMAG, C>([&](int i) { return unpack(r[(i / C) * (C + 1) + (i % C)]); }, st_,
                                       (size_t)warp * nx, nx, t, red + warp);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double N[3] = {red[0] * p.cell, red[1] * p.cell, red[2] * p.cell};
            const bool fin = isfinite(N[0]) && isfinite(N[1]) && isfinite(N[2]);
            finite = finite && fin;
            double d[3];
            renorm_factors(N, fin ? renorm : 0, p.mag, d);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                ds[j] = to_r<R>(d[j]);
                dlast[j] = d[j];
                sc->norms[j] = N[j];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 3 * nx; i += kStep1dThreads) A[i] = st_[i];
    if (threadIdx.x == 0 && nsteps > 0) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            sc->scale[j] = dlast[j];
            sc->scale_f[j] = (float)dlast[j];
            sc->scale_l[j] = (float)(dlast[j] - (double)sc->scale_f[j]);
        }
        sc->scale_src = 0;
        if (!finite) sc->err |= 1;
        sc->step_idx = step0 + nsteps;
    }
}

// ---------------------------------------------------------------------------
// CN along y: block = one warp solving K adjacent columns of one component
// (K = 2 for small chunks: a lane's chunk rows then load 32 contiguous bytes
// per row in FP64). Norm partials as for the x sweep, one slot per block.
// ---------------------------------------------------------------------------
// Columns [col, col + K) of component j of one grid by the calling warp; part
// (nullable) as for cnx_line.
template <typename R, bool IMAG, int C, typename P = double>
__device__ __forceinline__ void cny_cols(const typename V2<R>::T* in, typename V2<R>::T* out, const KParams& p,
                                         const Tabs<R>& t, int j, int col, P* part) {
    constexpr int K = CnShape<R, C>::K;
    constexpr bool KEEP = CnShape<R, C>::KEEP;
    constexpr bool INC = sizeof(R) == 4;
    const int lane = threadIdx.x & 31;
    const int n = p.ny;
    const int i0 = lane * C;
    const size_t base = (size_t)j * p.nx * p.ny;
    const cx<R> zero = {R(0), R(0)};
    LaneTabs<R, IMAG, C> lt;
    lt.init(t, i0);
    cx<R> x[K][KEEP ? C : 1], v[K][C];
#pragma unroll
    for (int m = 0; m < C; m++) {
        const bool ok = i0 + m < n;
        size_t g = base + (size_t)(i0 + m) * p.nx + col;
#pragma unroll
        for (int k = 0; k < K; k++) {
            v[k][m] = (ok && col + k < p.nx) ? ldc<R>(in, g + k) : zero;
            if (KEEP) x[k][m] = v[k][m];
        }
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
        if constexpr (INC) cn_increment_rhs<R, IMAG, C>(v[k], t);
        solve_chunk<R, IMAG, C>(v[k], lt);
    }
    // complex64: only the stores remain, let the next step kernel launch (the
    // FP64 form measured faster with the implicit trigger at completion)
    if (sizeof(R) == 4) pdl_trigger();
    NormAcc<R> acc;
#pragma unroll
    for (int m = 0; m < C; m++) {
        if (i0 + m < n) {
            size_t g = base + (size_t)(i0 + m) * p.nx + col;
#pragma unroll
            for (int k = 0; k < K; k++) {
                if (col + k < p.nx) {
                    cx<R> xm = KEEP ? x[k][m] : ldc<R>(in, g + k);
                    cx<R> o = INC ? cx<R>{fma(R(2), v[k][m].re, xm.re), fma(R(2), v[k][m].im, xm.im)}
                                  : cx<R>{fma(R(2), v[k][m].re, -xm.re), fma(R(2), v[k][m].im, -xm.im)};
                    st<R>(out, g + k, o);
                    if (part) acc.add(o);
                }
            }
        }
    }
    if (part) {
        const P t = warp_sum(acc_value<P>(acc));
        if (lane == 0) *part = t;
    }
}

// sc (nullable): the fused 2D step. With renorm != 0 its next head kernel
// derives the pending scale from these partials: block 0 marks that
// (DevScalars::scale_src); with renorm == 0 the pending scale is 1 from here on
// and block 0 stores it. If advance, block 0 also moves the step counter on (the
// head kernel of this step has finished).
template <typename R, bool IMAG, int C>
__global__ void __launch_bounds__(32) k_cny_reg(const typename V2<R>::T* in, typename V2<R>::T* out, KParams p,
                                                Tabs<R> t, double* partials, DevScalars* sc, int renorm,
                                                int advance) {
    constexpr int K = CnShape<R, C>::K;
    const int ncb = (p.nx + K - 1) / K;
    const int j = blockIdx.x / ncb;
    const int col = (blockIdx.x - j * ncb) * K;
    pdl_wait();
    if (sc && blockIdx.x == 0 && threadIdx.x < 3) {
        if (renorm) {
            if (threadIdx.x == 0) sc->scale_src = 1;
        } else {
            sc->scale[threadIdx.x] = 1.0;
            sc->scale_f[threadIdx.x] = 1.0f;
            sc->scale_l[threadIdx.x] = 0.0f;
        }
        if (advance && threadIdx.x == 0) sc->step_idx += 1;
    }
    using P = typename PartT<R>::T;
    P* parts = reinterpret_cast<P*>(partials);
    cny_cols<R, IMAG, C, P>(in, out, p, t, j, col, parts ? parts + blockIdx.x : nullptr);
}

// ---------------------------------------------------------------------------
// Crank-Nicolson sweeps for lines longer than 1024 points (Sec. 3 LU / LUX /
// LUY). A line of n points is held by a group of nw = ceil(n / 512) warps, 16
// points per lane (lane g = part * 32 + lane of the group owns points
// [16 g, 16 g + 16)), staged in shared memory in a padded chunk layout (stride
// 17: conflict-free chunk reads). Each lane runs the forward and backward
// recurrences of its chunk with the precomputed LU factors (chunk products fp,
// fq over 16-point chunks); the chunk maps are composed by shuffles inside each
// warp and then across the group's warps through shared memory, both
// compositions stopping once the composed factor is negligible (tiny_carry).
// ---------------------------------------------------------------------------
constexpr int kLongS = kLongC + 1;  // padded chunk stride (shared memory)
__device__ __forceinline__ int long_slot(int i) { return (i >> 4) * kLongS + (i & (kLongC - 1)); }

// Solve T w = x for the lane's chunk v (in: x, out: w) at points [16 g, 16 g + 16),
// g = part * 32 + lane, of a line held by the nw warps of a group; part: this
// warp's index in the group; seg: the group's shared scratch of 4 nw entries.
// The tables are lane-interleaved (k_coef): chunk entry m of lane g at m G + g,
// G = 32 nw. Every thread of the block must call this (block barriers inside).
template <typename R, bool IMAG>
__device__ __forceinline__ void group_solve(cx<R> (&v)[kLongC], const Tabs<R>& t, int part, int nw, cx<R>* seg) {
    const int lane = threadIdx.x & 31;
    const int G = 32 * nw, g = part * 32 + lane;
    const cx<R> zero = {R(0), R(0)};
    cx<R> y = zero;
#pragma unroll
    for (int m = 0; m < kLongC; m++) {
        y = tfma<IMAG>(tld<R>(t.fg, m * G + g), y, tmul<IMAG>(tld<R>(t.fa, m * G + g), v[m]));
        v[m] = y;
    }
    cx<R> A = tld<R>(t.fp, (kLongC - 1) * G + g), B = y;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const cx<R> Ap = shup(A, off), Bp = shup(B, off);
        if (lane >= off) {
            B = tfma<IMAG>(A, Bp, B);
            A = tmul<IMAG>(A, Ap);
        }
        if (scan_done(lane < 2 * off, A)) break;
    }
    if (lane == 31) {
        seg[part] = A;
        seg[nw + part] = B;
    }
    __syncthreads();
    // y at the last point of the group's earlier warps
    cx<R> cw = zero;
    if (part > 0) {
        cw = seg[nw + part - 1];
        cx<R> wgt = seg[part - 1];
        for (int r = part - 2; r >= 0; r--) {
            if (tiny_carry(wgt.re) && tiny_carry(wgt.im)) break;
            cw = tfma<IMAG>(wgt, seg[nw + r], cw);
            wgt = tmul<IMAG>(wgt, seg[r]);
        }
    }
    const cx<R> Au = shup(A, 1), Bu = shup(B, 1);
    const cx<R> cin = lane == 0 ? cw : tfma<IMAG>(Au, cw, Bu);
    cx<R> w = zero;
#pragma unroll
    for (int m = kLongC - 1; m >= 0; m--) {
        const cx<R> yi = tfma<IMAG>(tld<R>(t.fp, m * G + g), cin, v[m]);
        w = tfma<IMAG>(tld<R>(t.fg, m * G + g), w, yi);
        v[m] = w;
    }
    A = tld<R>(t.fq, g);
    B = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const cx<R> An = shdn(A, off), Bn = shdn(B, off);
        if (lane + off < 32) {
            B = tfma<IMAG>(A, Bn, B);
            A = tmul<IMAG>(A, An);
        }
        if (scan_done(lane + 2 * off >= 32, A)) break;
    }
    if (lane == 0) {
        seg[2 * nw + part] = A;
        seg[3 * nw + part] = B;
    }
    __syncthreads();
    // w at the first point of the group's later warps
    cx<R> cbw = zero;
    if (part + 1 < nw) {
        cbw = seg[3 * nw + part + 1];
        cx<R> wgt = seg[2 * nw + part + 1];
        for (int r = part + 2; r < nw; r++) {
            if (tiny_carry(wgt.re) && tiny_carry(wgt.im)) break;
            cbw = tfma<IMAG>(wgt, seg[3 * nw + r], cbw);
            wgt = tmul<IMAG>(wgt, seg[2 * nw + r]);
        }
    }
    const cx<R> An = shdn(A, 1), Bn = shdn(B, 1);
    const cx<R> cb = lane == 31 ? cbw : tfma<IMAG>(An, cbw, Bn);
#pragma unroll
    for (int m = 0; m < kLongC; m++) v[m] = tfma<IMAG>(tld<R>(t.fq, m * G + g), cb, v[m]);
}

// ---------------------------------------------------------------------------
// Constant-factor solve of a long line (Tabs::uks > 0). The coefficient is
// real in imaginary time and complex in real time; complex64 pairs go through
// the packed FP32x2 instructions (two FP32 operations each, rounded as the two
// scalar ones would be).
// ---------------------------------------------------------------------------
template <bool IMAG, typename R> struct UCoef { using T = cx<R>; };
template <typename R> struct UCoef<true, R> { using T = R; };
template <bool IMAG, typename R> __device__ __forceinline__ typename UCoef<IMAG, R>::T ucoef(cx<R> v) {
    if constexpr (IMAG)
        return v.re;
    else
        return v;
}
template <typename R> __device__ __forceinline__ cx<R> gcx(R a) { return cx<R>{a, R(0)}; }
template <typename R> __device__ __forceinline__ cx<R> gcx(cx<R> a) { return a; }
template <typename R> __device__ __forceinline__ R gzero(R) { return R(0); }
template <typename R> __device__ __forceinline__ cx<R> gzero(cx<R>) { return cx<R>{R(0), R(0)}; }
// g y + x
template <typename R> __device__ __forceinline__ cx<R> gfma(R g, cx<R> y, cx<R> x) { return axpy(g, y, x); }
template <typename R> __device__ __forceinline__ cx<R> gfma(cx<R> g, cx<R> y, cx<R> x) { return caxpy(g, y, x); }
template <typename R> __device__ __forceinline__ cx<R> gmul(R g, cx<R> y) { return scl(g, y); }
template <typename R> __device__ __forceinline__ cx<R> gmul(cx<R> g, cx<R> y) { return mul(g, y); }
template <typename R> __device__ __forceinline__ R gprod(R a, R b) { return a * b; }
template <typename R> __device__ __forceinline__ cx<R> gprod(cx<R> a, cx<R> b) { return mul(a, b); }
// g y - x
template <typename R> __device__ __forceinline__ cx<R> gfms(R g, cx<R> y, cx<R> x) {
    return {fma(g, y.re, -x.re), fma(g, y.im, -x.im)};
}
template <typename R> __device__ __forceinline__ cx<R> gfms(cx<R> g, cx<R> y, cx<R> x) {
    return caxpy(g, y, cx<R>{-x.re, -x.im});
}
template <typename R> __device__ __forceinline__ cx<R> gadd(cx<R> a, cx<R> b) { return add(a, b); }
template <typename R> __device__ __forceinline__ cx<R> gsub(cx<R> a, cx<R> b) { return sub(a, b); }
template <typename R> __device__ __forceinline__ R gshup(R a, int off) { return shfl_up_r(a, off); }
template <typename R> __device__ __forceinline__ cx<R> gshup(cx<R> a, int off) { return shup(a, off); }
template <typename R> __device__ __forceinline__ R gshdn(R a, int off) { return shfl_dn_r(a, off); }
template <typename R> __device__ __forceinline__ cx<R> gshdn(cx<R> a, int off) { return shdn(a, off); }
template <typename R> __device__ __forceinline__ bool gtiny(R a) { return tiny_carry(a); }
template <typename R> __device__ __forceinline__ bool gtiny(cx<R> a) { return tiny_carry(a.re) && tiny_carry(a.im); }
__device__ __forceinline__ float2 f2(cx<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ cx<float> fc(float2 a) { return cx<float>{a.x, a.y}; }
__device__ __forceinline__ cx<float> gfma(float g, cx<float> y, cx<float> x) {
    return fc(__ffma2_rn(make_float2(g, g), f2(y), f2(x)));
}
__device__ __forceinline__ cx<float> gmul(float g, cx<float> y) { return fc(__fmul2_rn(make_float2(g, g), f2(y))); }
__device__ __forceinline__ cx<float> gadd(cx<float> a, cx<float> b) { return fc(__fadd2_rn(f2(a), f2(b))); }
// a - b = fma(b, -1, a), exactly rounded once
__device__ __forceinline__ cx<float> gsub(cx<float> a, cx<float> b) {
    return fc(__ffma2_rn(f2(b), make_float2(-1.0f, -1.0f), f2(a)));
}
// pw y + x with a chunk carry weight pw (Tabs::upow: in imaginary time the
// real power in both halves, which complex64 uses as the packed pair)
template <bool IMAG, typename R> __device__ __forceinline__ cx<R> pfma(cx<R> pw, cx<R> y, cx<R> x) {
    if constexpr (IMAG && std::is_same<R, float>::value)
        return fc(__ffma2_rn(f2(pw), f2(y), f2(x)));
    else if constexpr (IMAG)
        return axpy(pw.re, y, x);
    else
        return caxpy(pw, y, x);
}
__device__ __forceinline__ double shfl0(double v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ float shfl0(float v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ df shfl0(df v) {
    return df(__shfl_sync(0xffffffffu, v.hi, 0), __shfl_sync(0xffffffffu, v.lo, 0));
}

// Solve the lane's chunk v (in: the right-hand side r of its 16 points i0 ..
// i0 + 15; out: q = w / ua with T w = r) for the group's line of n points.
// Forward z_i = r_i + g z_(i-1), backward q_i = z_i + g q_(i+1) with the same
// chunk scans and cross-warp carries as group_solve; a chunk that reaches past n
// has the chunk factor 0 and zeros past n (the tables hold fg = 0 there), and
// the first unks points take the correction of the first diagonal entry.
template <typename R, bool IMAG>
__device__ __forceinline__ void group_solve_uni(cx<R> (&v)[kLongC], const Tabs<R>& t, int part, int nw, cx<R>* seg,
                                                int n, int i0) {
    using G = typename UCoef<IMAG, R>::T;
    const int lane = threadIdx.x & 31;
    const cx<R> zero = {R(0), R(0)};
    const G g = ucoef<IMAG>(t.ug), g16 = ucoef<IMAG>(t.ug16), gz = gzero(g);
    const bool full = i0 + kLongC <= n;
    const int nlev = t.unlev;
    cx<R> z = zero;
#pragma unroll
    for (int m = 0; m < kLongC; m++) {
        z = gfma(g, z, v[m]);
        v[m] = z;
    }
    G A = full ? g16 : gz;
    cx<R> B = full ? z : zero;
    for (int l = 0, off = 1; l < nlev; l++, off <<= 1) {
        const G Ap = gshup(A, off);
        const cx<R> Bp = shup(B, off);
        if (lane >= off) {
            B = gfma(A, Bp, B);
            A = gprod(A, Ap);
        }
    }
    if (lane == 31) {
        seg[part] = gcx(A);
        seg[nw + part] = B;
    }
    __syncthreads();
    cx<R> cw = zero;
    if (part > 0) {
        cw = seg[nw + part - 1];
        G wgt = ucoef<IMAG>(seg[part - 1]);
        for (int r = part - 2; r >= 0; r--) {
            if (gtiny(wgt)) break;
            cw = gfma(wgt, seg[nw + r], cw);
            wgt = gprod(wgt, ucoef<IMAG>(seg[r]));
        }
    }
    {
        const G Au = gshup(A, 1);
        const cx<R> Bu = shup(B, 1);
        const cx<R> cin = lane == 0 ? cw : gfma(Au, cw, Bu);
        // z_m += g^(m+1) cin
#pragma unroll
        for (int m = 0; m < kLongC; m++) v[m] = pfma<IMAG>(t.upow[m], cin, v[m]);
    }
    if (!full) {
#pragma unroll
        for (int m = 0; m < kLongC; m++)
            if (i0 + m >= n) v[m] = zero;
    }
    cx<R> q = zero;
#pragma unroll
    for (int m = kLongC - 1; m >= 0; m--) {
        q = gfma(g, q, v[m]);
        v[m] = q;
    }
    A = full ? g16 : gz;
    B = q;
    for (int l = 0, off = 1; l < nlev; l++, off <<= 1) {
        const G An = gshdn(A, off);
        const cx<R> Bn = shdn(B, off);
        if (lane + off < 32) {
            B = gfma(A, Bn, B);
            A = gprod(A, An);
        }
    }
    if (lane == 0) {
        seg[2 * nw + part] = gcx(A);
        seg[3 * nw + part] = B;
    }
    __syncthreads();
    cx<R> cbw = zero;
    if (part + 1 < nw) {
        cbw = seg[3 * nw + part + 1];
        G wgt = ucoef<IMAG>(seg[2 * nw + part + 1]);
        for (int r = part + 2; r < nw; r++) {
            if (gtiny(wgt)) break;
            cbw = gfma(wgt, seg[3 * nw + r], cbw);
            wgt = gprod(wgt, ucoef<IMAG>(seg[2 * nw + r]));
        }
    }
    {
        const G An = gshdn(A, 1);
        const cx<R> Bn = shdn(B, 1);
        const cx<R> cb = lane == 31 ? cbw : gfma(An, cbw, Bn);
        // q_m += g^(16 - m) cb
#pragma unroll
        for (int m = 0; m < kLongC; m++) v[m] = pfma<IMAG>(t.upow[kLongC - 1 - m], cb, v[m]);
    }
    if (part == 0) {
        const cx<R> q0 = {shfl0(v[0].re), shfl0(v[0].im)};
        if (i0 < t.uks) {
            const cx<R> cq = mul(t.uc, q0);
#pragma unroll
            for (int m = 0; m < kLongC; m++)
                if (i0 + m < t.uks) v[m] = sub(v[m], mul(cq, tld<R>(t.us, i0 + m)));
        }
    }
}

// Per-lane |o|^2 sum of the complex64 state on the packed FP32x2 instructions:
// the same error-free square split and two-sum as NormAcc<float>, with the real
// and imaginary squares in the two halves.
struct NormAccF2 {
    float2 hi = {0.0f, 0.0f}, lo = {0.0f, 0.0f};
    __device__ __forceinline__ void add(cx<float> o) {
        const float2 m1 = make_float2(-1.0f, -1.0f);
        const float2 x = f2(o);
        const float2 p = __fmul2_rn(x, x);
        const float2 e = __ffma2_rn(x, x, __fmul2_rn(p, m1));
        const float2 s = __fadd2_rn(hi, p);
        const float2 bp = __ffma2_rn(hi, m1, s);
        const float2 r = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, m1, s), m1, hi), __ffma2_rn(bp, m1, p));
        lo = __fadd2_rn(lo, __fadd2_rn(r, e));
        hi = s;
    }
    __device__ __forceinline__ df dfvalue() const {
        return fast_two_sum(hi.x, lo.x) + fast_two_sum(hi.y, lo.y);
    }
};

// The constant-factor variant of long_line (below): the right-hand side is
// L x (increment form) or x, the solve gives q, and the result is x + uk q or
// uk q - x.
template <typename R, bool IMAG>
__device__ __forceinline__ typename PartT<R>::T long_line_uni(cx<R>* line, int n, const Tabs<R>& t, int part, int nw,
                                                              cx<R>* seg, bool want_norm = true) {
    const int i0 = (part * 32 + (threadIdx.x & 31)) * kLongC;
    constexpr bool INC = sizeof(R) == 4;
    const cx<R> zero = {R(0), R(0)};
    cx<R> v[kLongC];
#pragma unroll
    for (int m = 0; m < kLongC; m++) v[m] = line[long_slot(i0 + m)];
    if constexpr (INC) {
        cx<R> prev = i0 > 0 ? line[long_slot(i0 - 1)] : zero;
        const cx<R> last = i0 + kLongC < n ? line[long_slot(i0 + kLongC)] : zero;
#pragma unroll
        for (int m = 0; m < kLongC; m++) {
            const cx<R> cur = v[m];
            const cx<R> nxt = m + 1 < kLongC ? v[m + 1] : last;
            v[m] = i0 + m < n ? gadd(gsub(prev, cur), gsub(nxt, cur)) : zero;
            prev = cur;
        }
    }
    group_solve_uni<R, IMAG>(v, t, part, nw, seg, n, i0);
    const auto k = ucoef<IMAG>(t.uk);
    typename std::conditional<INC && IMAG, NormAccF2, NormAcc<R>>::type acc;
    auto result = [&](int m) {
        const cx<R> x = line[long_slot(i0 + m)];
        cx<R> o;
        if constexpr (INC)
            o = gfma(k, v[m], x);
        else
            o = gfms(k, v[m], x);
        line[long_slot(i0 + m)] = o;
        return o;
    };
    if (want_norm) {
#pragma unroll
        for (int m = 0; m < kLongC; m++)
            if (i0 + m < n) acc.add(result(m));
    } else {
        // (points past n: their slots are never stored)
#pragma unroll
        for (int m = 0; m < kLongC; m++) result(m);
    }
    if constexpr (INC && IMAG)
        return acc.dfvalue();
    else
        return acc_value<typename PartT<R>::T>(acc);
}

// The sweep of one staged line: lane chunk in from shared memory (line, padded
// layout), solve, and the result o written back to the lane's own slots.
// complex64: increment form o = x + 2 e, T e = bt L x (the differences of
// neighbouring values exact); otherwise o = 2 w - x. Returns |o|^2 summed over
// the lane's points (for the norm partials).
template <typename R, bool IMAG, bool UNI>
__device__ __forceinline__ typename PartT<R>::T long_line(cx<R>* line, int n, const Tabs<R>& t, int part, int nw,
                                                          cx<R>* seg, bool want_norm = true) {
    if constexpr (UNI) return long_line_uni<R, IMAG>(line, n, t, part, nw, seg, want_norm);
    const int i0 = (part * 32 + (threadIdx.x & 31)) * kLongC;
    constexpr bool INC = sizeof(R) == 4;
    const cx<R> zero = {R(0), R(0)};
    cx<R> v[kLongC];
#pragma unroll
    for (int m = 0; m < kLongC; m++) v[m] = line[long_slot(i0 + m)];
    if constexpr (INC) {
        const cx<R> a0 = tld<R>(t.fa, 0), g0 = tld<R>(t.fg, 0);
        cx<R> bt;
        if (IMAG) {
            bt = {g0.re / a0.re, R(0)};
        } else {
            const R den = nrm(a0);
            const cx<R> q = cmul(a0, g0);  // conj(a0) g0
            bt = {q.re / den, q.im / den};
        }
        cx<R> prev = i0 > 0 ? line[long_slot(i0 - 1)] : zero;
        const cx<R> last = i0 + kLongC < n ? line[long_slot(i0 + kLongC)] : zero;
#pragma unroll
        for (int m = 0; m < kLongC; m++) {
            const cx<R> cur = v[m];
            const cx<R> nxt = m + 1 < kLongC ? v[m + 1] : last;
            v[m] = i0 + m < n ? tmul<IMAG>(bt, add(sub(prev, cur), sub(nxt, cur))) : zero;
            prev = cur;
        }
    }
    group_solve<R, IMAG>(v, t, part, nw, seg);
    NormAcc<R> acc;
#pragma unroll
    for (int m = 0; m < kLongC; m++) {
        if (i0 + m < n) {
            const cx<R> x = line[long_slot(i0 + m)];
            const cx<R> o = INC ? cx<R>{fma(R(2), v[m].re, x.re), fma(R(2), v[m].im, x.im)}
                                : cx<R>{fma(R(2), v[m].re, -x.re), fma(R(2), v[m].im, -x.im)};
            line[long_slot(i0 + m)] = o;
            acc.add(o);
        }
    }
    return acc_value<typename PartT<R>::T>(acc);
}

// The block's norm partial from each thread's lane sum v (every thread of the
// block calls it; fixed order: warps by shuffles, then the warps in index
// order by thread 0, which returns the sum). FP64 for complex128, a
// double-float pair on the FP32 pipe otherwise.
template <typename P> __device__ __forceinline__ P block_part(P v, P* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    P s = red[0];
    if (threadIdx.x == 0)
        for (int w = 1; w < nw; w++) s = s + red[w];
    return s;
}

// CN along x for lines of 1025..8192 points: one block of nw warps per line
// (line l = j*ny + iy, row iy of component j). in may equal out. With part
// non-null (1D: the step's last pass) the block writes the norm of its line to
// part[line] (PartT<R>: FP64 for complex128, a double-float pair otherwise).
// UNI: the constant-factor solve (Tabs::uks > 0; complex64 and double-float)
// instead of the tables; the two are separate instantiations so that neither
// carries the other's registers.
template <typename R, bool UNI> constexpr int long_min_blocks() { return (UNI && sizeof(R) == 4) ? 2 : 1; }

template <typename R, bool IMAG, bool UNI>
__global__ void __launch_bounds__(32 * kLongMaxWarps, long_min_blocks<R, UNI>())
    k_cn_x(const typename V2<R>::T* in, typename V2<R>::T* out,
                                                             KParams p, Tabs<R> t, double* part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* line = reinterpret_cast<cx<R>*>(smem_raw);
    using P = typename PartT<R>::T;
    __shared__ cx<R> seg[4 * kLongMaxWarps];
    __shared__ P red[kLongMaxWarps];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const int n = p.nx;
    const size_t base = (size_t)blockIdx.x * n;
    // the block's 32 nw threads stage the span = 16 * 32 nw points: all 16 loads of a
    // thread in flight before the shared-memory stores. Point threadIdx.x + k blockDim
    // sits at slot long_slot(threadIdx.x) + k sstep (blockDim is a multiple of 16).
    const int sstep = ((int)blockDim.x >> 4) * kLongS;
    const typename V2<R>::T* src = in + base + threadIdx.x;
    typename V2<R>::T* dst = out + base + threadIdx.x;
    cx<R>* slot = line + long_slot(threadIdx.x);
    const int rem = n - (int)threadIdx.x;  // point k is in the line when k blockDim < rem
    pdl_wait();
    {
        cx<R> tmp[kLongC];
#pragma unroll
        for (int k = 0; k < kLongC; k++)
            tmp[k] = k * (int)blockDim.x < rem ? ldc<R>(src, (size_t)k * blockDim.x) : cx<R>{R(0), R(0)};
#pragma unroll
        for (int k = 0; k < kLongC; k++) slot[k * sstep] = tmp[k];
    }
    __syncthreads();
    const P acc = long_line<R, IMAG, UNI>(line, n, t, warp, nw, seg, part != nullptr);
    pdl_trigger();  // the next sweep's blocks may take the slots this grid frees
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kLongC; k++)
        if (k * (int)blockDim.x < rem) st<R>(dst, (size_t)k * blockDim.x, slot[k * sstep]);
    if (part) {
        const P sum = block_part(acc, red);
        if (threadIdx.x == 0) reinterpret_cast<P*>(part)[blockIdx.x] = sum;
    }
}

constexpr int kPwxLongMaxGroupWarps = 4;
// The row iy of k_pwx_long once the pending scale ds and Omega are known: the
// point pairs into the three lines' chunk layout in shared memory, the three line
// solves by the block's warp groups (blockDim = 96 nwl), the lines to B. Every
// thread of the block calls it.
template <bool IMAG, bool STD>
__device__ __forceinline__ void pwx_long_row(const float2* __restrict__ A, float2* __restrict__ B, const KParams& p,
                                             const f32x2 (&ds)[3], float Ot, const Tabs<float>& t, int mask, int iy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<float>* lines = reinterpret_cast<cx<float>*>(smem_raw);  // [3][32 nwl kLongS]
    __shared__ cx<float> seg[3][4 * kPwxLongMaxGroupWarps];
    const int nwl = blockDim.x / 96;
    const int warp = threadIdx.x >> 5;
    const int nx = p.nx;
    const int span = 32 * kLongC * nwl, S = 32 * nwl * kLongS;
    for (int q = threadIdx.x; 2 * q < nx; q += blockDim.x) {
        cx<f32x2> u[3];
        pair_substeps<IMAG, STD>(A, p, ds, Ot, mask, 2 * q, iy, u);
        const int s0 = long_slot(2 * q);  // 2q is even: 2q + 1 sits in the next slot of the same chunk
#pragma unroll
        for (int j = 0; j < 3; j++) {
            lines[j * S + s0] = cx<float>{u[j].re.v.x, u[j].im.v.x};
            lines[j * S + s0 + 1] = cx<float>{u[j].re.v.y, u[j].im.v.y};
        }
    }
    for (int i = nx + threadIdx.x; i < span; i += blockDim.x)
#pragma unroll
        for (int j = 0; j < 3; j++) lines[j * S + long_slot(i)] = cx<float>{0.0f, 0.0f};
    __syncthreads();
    const int j = warp / nwl;
    long_line_uni<float, IMAG>(lines + j * S, nx, t, warp - j * nwl, nwl, seg[j], false);
    pdl_trigger();  // the y sweep's blocks may take the slots this grid frees
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float2* dst = B + ((size_t)c * p.ny + iy) * nx;
        const cx<float>* src = lines + c * S;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) dst[i] = make_float2(src[long_slot(i)].re, src[long_slot(i)].im);
    }
}

// Pointwise substeps and CN along x of one row of a 2D complex64 grid with even
// rows of at most 2048 points (1025..2048, or the rows of a tiled grid; the
// constant-factor solve, Tabs::uks > 0): one block per row, 3 groups of nwl =
// ceil(nx / 512) warps (one group per component line). The threads evaluate the
// row's point pairs (pair_substeps) into the padded chunk layout of the three
// lines in shared memory (slots past nx zero), then group j solves line j
// (long_line_uni) and the block stores the three lines to B. Each step then
// streams the state twice (A -> B here, B -> A in the y sweep) instead of three
// times. With partials (the tiled step) every block first forms the pending
// scale from the previous y tiles' norm partials, as k_pwx does.
template <bool IMAG, bool STD>
__global__ void __launch_bounds__(96 * kPwxLongMaxGroupWarps, 2)
    k_pwx_long(const float2* __restrict__ A, float2* __restrict__ B, KParams p, const DevScalars* __restrict__ sc,
               const double* __restrict__ omega_tab, Tabs<float> t, int mask, const double* __restrict__ partials,
               int m, int renorm) {
    __shared__ df red_df[3];
    __shared__ float dsh[3];
    const int warp = threadIdx.x >> 5;
    const int iy = blockIdx.x;
    pdl_wait();
    f32x2 ds[3];
    float Ot;
    pair_constants(p, sc, omega_tab, mask, ds, Ot);
    if (partials && *(volatile const int*)&sc->scale_src) {
        // the previous y sweep left its norm partials (m per component, double-float
        // pairs): every block forms the pending scale from them, in the same order
        if (warp < 3) {
            const df sm = sum_partials_warp(reinterpret_cast<const df*>(partials) + (size_t)warp * m, m);
            if ((threadIdx.x & 31) == 0) red_df[warp] = sm;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const df S3[3] = {red_df[0], red_df[1], red_df[2]};
            df f[3];
            double d[3], N[3];
            bool finite;
            scale_from_df_sums(S3, p.cell, renorm, p.mag, f, d, N, finite);
#pragma unroll
            for (int j = 0; j < 3; j++) dsh[j] = to_r_df<float>(f[j]);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 3; j++) ds[j] = f32x2(dsh[j]);
    }
    pwx_long_row<IMAG, STD>(A, B, p, ds, Ot, t, mask, iy);
}

// CN along y for columns of 1025..8192 points: one block per tile of kc (1, 2
// or 4) adjacent columns [col0, col0 + kc) of component j, staged in shared memory (row
// segments of kc elements), nw warps per column. With part non-null the block
// writes the norm of its tile to part[blockIdx.x] (the blocks of component j are
// contiguous; PartT<R> as for k_cn_x).
template <typename R, bool IMAG, bool UNI>
__global__ void __launch_bounds__(32 * kLongMaxWarps, long_min_blocks<R, UNI>())
    k_cn_y(const typename V2<R>::T* in, typename V2<R>::T* out,
                                                             KParams p, Tabs<R> t, int kc, double* part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using P = typename PartT<R>::T;
    __shared__ cx<R> seg[4 * kLongMaxWarps];
    __shared__ P red[kLongMaxWarps];
    const int warp = threadIdx.x >> 5;
    const int nw = (blockDim.x >> 5) / kc;
    const int n = p.ny, span = 32 * kLongC * nw;
    const int ncb = (p.nx + kc - 1) / kc;
    const int j = blockIdx.x / ncb;
    const int col0 = (blockIdx.x - j * ncb) * kc;
    const size_t base = (size_t)j * p.nx * p.ny;
    cx<R>* lines = reinterpret_cast<cx<R>*>(smem_raw);  // [kc][span padded]
    // complex64 tiles of 4 columns: the columns start 4 elements (4 bank pairs) apart
    // modulo 16, so the threads that stage one row segment use different banks
    const size_t lstride = (size_t)(span / kLongC) * kLongS + long_col_pad(sizeof(cx<R>), kc);
    const int lkc = kc == 4 ? 2 : kc == 2 ? 1 : 0;  // kc is 1, 2 or 4
    // thread -> (row it0 + k rs, column cc) of the tile: blockDim is a multiple of
    // 16 kc, so rs = blockDim / kc is a multiple of 16 and the padded slot of row
    // it0 + k rs is long_slot(it0) + k (rs / 16) kLongS
    const int cc = threadIdx.x & (kc - 1), it0 = threadIdx.x >> lkc, rs = blockDim.x >> lkc;
    const int col = col0 + cc, sstep = (rs >> 4) * kLongS;
    const bool colok = col < p.nx;
    const size_t gstep = (size_t)rs * p.nx;
    cx<R>* tcol = lines + cc * lstride + long_slot(it0);
    // the block's 32 nw kc threads stage span * kc = 16 * blockDim values: all 16 loads
    // of a thread in flight before the shared-memory stores
    {
        cx<R> tmp[kLongC];
        size_t g = base + (size_t)it0 * p.nx + col;
#pragma unroll
        for (int k = 0; k < kLongC; k++, g += gstep)
            tmp[k] = (it0 + k * rs < n && colok) ? ldc<R>(in, g) : cx<R>{R(0), R(0)};
#pragma unroll
        for (int k = 0; k < kLongC; k++) tcol[k * sstep] = tmp[k];
    }
    __syncthreads();
    const int c = warp / nw;
    P acc = long_line<R, IMAG, UNI>(lines + c * lstride, n, t, warp - c * nw, nw, seg + 4 * nw * c);
    __syncthreads();
    if (colok) {
        size_t g = base + (size_t)it0 * p.nx + col;
        const cx<R>* src = tcol;
        for (int i = it0; i < n; i += rs, g += gstep, src += sstep) st<R>(out, g, *src);
    }
    if (part) {
        if (col0 + c >= p.nx) acc = P(0);
        const P sum = block_part(acc, red);
        if (threadIdx.x == 0) reinterpret_cast<P*>(part)[blockIdx.x] = sum;
    }
}


// ---------------------------------------------------------------------------
// CN along y in row tiles, for the constant-factor solve (Tabs::uks > 0) when
// a chunk's carries reach at most kTileMaxHalo chunks: |g^16|^hc < 2^-64 (the
// small bt of the workloads, where g = bt / u is about 0.02). A block holds
// a tile of 32 adjacent columns, one per lane, so that every warp load and
// store is one contiguous row segment (256 bytes in complex64), and the rows
// [y0 - 16 hc, y0 + 16 (kTileReal + hc)): kTileReal chunks of 16 rows that it
// writes, and hc chunks above and below that only feed their carries. Warp w
// holds the chunk of rows i0 = y0 + 16 (w - hc) .. i0 + 15 of its lane's
// column in registers; the forward and backward carries of the hc nearest
// chunks are composed through shared memory (a chunk further away weighs less
// than 2^-64). The top tile applies the start correction of the first uks
// rows (uks <= 16 kTileReal). The arithmetic per point is that of
// long_line_uni. in != out: the halos read other tiles' input rows.
// ---------------------------------------------------------------------------

template <typename R, int HC, int RT = kTileReal> constexpr int tile_min_blocks() {
    return RT == kTileReal ? (sizeof(R) == 4 ? (HC == 1 ? 3 : 2) : 1) : (sizeof(R) == 4 ? (HC == 1 ? 5 : 4) : 2);
}

// One tile of the row-tiled y sweep: columns [32 ct, 32 ct + 32) of component j,
// rows [128 rt, 128 rt + 128) written (see k_cn_y_tile). Every thread of the block
// calls it after the dependency wait; with want_norm it returns the tile's |o|^2
// sum in thread 0 (PartT<R>), otherwise zero.
template <typename R, bool IMAG, int HC, int RT = kTileReal>
__device__ __forceinline__ typename PartT<R>::T cny_tile(const typename V2<R>::T* __restrict__ in,
                                                         typename V2<R>::T* __restrict__ out, const KParams& p,
                                                         const Tabs<R>& t, int j, int ct, int rt, bool want_norm) {
    using G = typename UCoef<IMAG, R>::T;
    using P = typename PartT<R>::T;
    using T = typename V2<R>::T;
    constexpr bool INC = sizeof(R) == 4;
    constexpr int NW = RT + 2 * HC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* xs = reinterpret_cast<cx<R>*>(smem_raw);  // [warp][m][lane]: the loaded values
    __shared__ cx<R> fend[NW][32], bend[NW][32];      // chunk ends of the two passes
    __shared__ cx<R> q0s[32];
    __shared__ P red[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = p.ny, nx = p.nx;
    const int y0 = rt * kLongC * RT, i0 = y0 + 16 * (w - HC);
    const int col = ct * 32 + lane;
    const bool colok = col < nx;
    // a lane past the last column reads column nx - 1 (in bounds) and stores nothing:
    // the columns are independent
    const size_t cbase = (size_t)j * nx * n + (colok ? col : nx - 1);
    const cx<R> zero = {R(0), R(0)};
    cx<R>* xw = xs + (size_t)w * kLongC * 32 + lane;
    // warp-uniform: the chunk and the rows next to it lie inside the column
    const bool inner = i0 >= 1 && i0 + kLongC < n;
    const T* src = in + cbase + (ptrdiff_t)i0 * nx;
    cx<R> v[kLongC];
    // the chunk's values x (kept in shared memory for the result) and the right-hand
    // side: L x (increment form) or x. IN: no row checks (inner chunk).
    auto load_rhs = [&](auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;
        cx<R> x[kLongC];
        cx<R> prev, last;
        if constexpr (IN) {
#pragma unroll
            for (int m = 0; m < kLongC; m++) x[m] = ldc<R>(src, (size_t)m * nx);
            prev = ldc<R>(src - nx, 0);
            last = ldc<R>(src, (size_t)kLongC * nx);
        } else {
#pragma unroll
            for (int m = 0; m < kLongC; m++) {
                const int i = i0 + m;
                x[m] = (i >= 0 && i < n) ? ldc<R>(in, cbase + (size_t)i * nx) : zero;
            }
            // the neighbours of the chunk's end rows (outside the tile they count as
            // zero: they feed the halo's carries only)
            const int im = i0 - 1, ip = i0 + kLongC;
            prev = (im >= 0 && im < n) ? ldc<R>(in, cbase + (size_t)im * nx) : zero;
            last = (ip >= 0 && ip < n) ? ldc<R>(in, cbase + (size_t)ip * nx) : zero;
        }
        if constexpr (INC) {
            // L x, zero outside the column
#pragma unroll
            for (int m = 0; m < kLongC; m++) {
                const cx<R> cur = x[m];
                const cx<R> nxt = m + 1 < kLongC ? x[m + 1] : last;
                const cx<R> r = gadd(gsub(prev, cur), gsub(nxt, cur));
                if constexpr (IN)
                    v[m] = r;
                else
                    v[m] = (i0 + m >= 0 && i0 + m < n) ? r : zero;
                prev = cur;
            }
        } else {
#pragma unroll
            for (int m = 0; m < kLongC; m++) v[m] = x[m];
        }
#pragma unroll
        for (int m = 0; m < kLongC; m++) xw[m * 32] = x[m];
    };
    if (inner)
        load_rhs(std::true_type{});
    else
        load_rhs(std::false_type{});
    const G g = ucoef<IMAG>(t.ug), g16 = ucoef<IMAG>(t.ug16);
    // forward z_i = r_i + g z_(i-1): the chunk from a zero start, then the carry
    cx<R> z = zero;
#pragma unroll
    for (int m = 0; m < kLongC; m++) {
        z = gfma(g, z, v[m]);
        v[m] = z;
    }
    fend[w][lane] = z;
    __syncthreads();
    {
        cx<R> cin = zero;
#pragma unroll
        for (int k = HC; k >= 1; k--)
            if (w - k >= 0) cin = gfma(g16, cin, fend[w - k][lane]);
        // z_m += g^(m+1) cin
#pragma unroll
        for (int m = 0; m < kLongC; m++) v[m] = pfma<IMAG>(t.upow[m], cin, v[m]);
    }
    if (i0 + kLongC > n) {
#pragma unroll
        for (int m = 0; m < kLongC; m++)
            if (i0 + m >= n) v[m] = zero;
    }
    // backward q_i = z_i + g q_(i+1)
    cx<R> q = zero;
#pragma unroll
    for (int m = kLongC - 1; m >= 0; m--) {
        q = gfma(g, q, v[m]);
        v[m] = q;
    }
    bend[w][lane] = q;
    __syncthreads();
    {
        cx<R> cb = zero;
#pragma unroll
        for (int k = HC; k >= 1; k--)
            if (w + k < NW) cb = gfma(g16, cb, bend[w + k][lane]);
        // q_m += g^(16 - m) cb
#pragma unroll
        for (int m = 0; m < kLongC; m++) v[m] = pfma<IMAG>(t.upow[kLongC - 1 - m], cb, v[m]);
    }
    if (y0 == 0) {  // the start correction: rows i < uks (block-uniform branch)
        if (w == HC) q0s[lane] = v[0];
        __syncthreads();
        if (w >= HC && i0 < t.uks) {
            const cx<R> cq = mul(t.uc, q0s[lane]);
#pragma unroll
            for (int m = 0; m < kLongC; m++)
                if (i0 + m < t.uks) v[m] = sub(v[m], mul(cq, tld<R>(t.us, i0 + m)));
        }
    }
    const auto k = ucoef<IMAG>(t.uk);
    typename std::conditional<INC && IMAG, NormAccF2, NormAcc<R>>::type acc;
    if (w >= HC && w < HC + RT && colok) {
        T* dst = out + cbase + (ptrdiff_t)i0 * nx;
        auto result = [&](int m) {
            const cx<R> x = xw[m * 32];
            cx<R> o;
            if constexpr (INC)
                o = gfma(k, v[m], x);
            else
                o = gfms(k, v[m], x);
            st<R>(dst, (size_t)m * nx, o);
            acc.add(o);
        };
        if (i0 + kLongC <= n) {
#pragma unroll
            for (int m = 0; m < kLongC; m++) result(m);
        } else {
#pragma unroll
            for (int m = 0; m < kLongC; m++)
                if (i0 + m < n) result(m);
        }
    }
    if (!want_norm) return P(0);
    P a;
    if constexpr (INC && IMAG)
        a = acc.dfvalue();
    else
        a = acc_value<P>(acc);
    return block_part(a, red);
}


// sc (nullable): the tiled step whose next head kernel forms the pending scale from
// these partials (as k_cny_reg: block 0 marks that, or stores the scale 1 when
// renorm == 0, and moves the step counter on if advance).
template <typename R, bool IMAG, int HC, int RT>
__global__ void __launch_bounds__(32 * (RT + 2 * HC), (tile_min_blocks<R, HC, RT>()))
    k_cn_y_tile(const typename V2<R>::T* __restrict__ in, typename V2<R>::T* __restrict__ out, KParams p, Tabs<R> t,
                double* part, DevScalars* sc, int renorm, int advance) {
    using P = typename PartT<R>::T;
    const int nrt = (p.ny + kLongC * RT - 1) / (kLongC * RT), nct = (p.nx + 31) >> 5;
    const int rt = blockIdx.x % nrt, rest = blockIdx.x / nrt;
    const int ct = rest % nct, j = rest / nct;
    pdl_wait();
    // with norm partials and no head scale the next launch is the finalize block, which
    // may become resident now (it waits for this grid); otherwise the next kernel
    // launches at the end
    if (part && !sc) pdl_trigger();
    if (sc && blockIdx.x == 0 && threadIdx.x < 3) {
        if (renorm) {
            if (threadIdx.x == 0) sc->scale_src = 1;
        } else {
            sc->scale[threadIdx.x] = 1.0;
            sc->scale_f[threadIdx.x] = 1.0f;
            sc->scale_l[threadIdx.x] = 0.0f;
        }
        if (advance && threadIdx.x == 0) sc->step_idx += 1;
    }
    const P sum = cny_tile<R, IMAG, HC, RT>(in, out, p, t, j, ct, rt, part != nullptr);
    if (part && threadIdx.x == 0) reinterpret_cast<P*>(part)[blockIdx.x] = sum;
}

}  // namespace sgpe
