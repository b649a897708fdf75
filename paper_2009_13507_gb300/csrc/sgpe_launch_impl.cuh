// sgpe_launch_impl.cuh -- launchers of the step / observable kernels for one
// storage precision; included once per precision translation unit.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>
#include "sgpe_cn.cuh"
#include "sgpe_kernels.cuh"
#include "sgpe_launch.h"
#include "sgpe_socn.cuh"
#include "sgpe_step1d_cl.cuh"

namespace sgpe {

// The constant-factor form serves the forms on the FP32 pipe; complex128 keeps
// the tables (their loads cost nothing next to its FP64 arithmetic, measured).
template <typename R> constexpr bool kUniForm = !std::is_same<R, double>::value;

template <typename R> static Tabs<R> make_tabs(const void* const* t) {
    using T = typename V2<R>::T;
    Tabs<R> r{};
    r.fa = (const T*)t[0];
    r.fg = (const T*)t[1];
    r.fp = (const T*)t[2];
    r.fq = (const T*)t[3];
    r.uks = 0;
    r.unlev = 5;
    return r;
}

static inline double2 pack_host(cx<double> a) { return make_double2(a.re, a.im); }
static inline float2 pack_host(cx<float> a) { return make_float2(a.re, a.im); }
static inline float4 pack_host(cx<df> a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
// A host double pair as the device complex type R (double-float: hi + lo split).
template <typename R> static cx<R> host_cx(double re, double im) { return cx<R>{(R)re, (R)im}; }
template <> cx<df> host_cx<df>(double re, double im) { return cx<df>{df_from(re), df_from(im)}; }
template <typename R> static typename V2<R>::T host_elem(double re, double im) { return pack_host(host_cx<R>(re, im)); }

template <typename R> static Tabs<R> make_tabs(const TabSet& ts) {
    Tabs<R> r = make_tabs<R>((const void* const*)ts.t);
    const UniHost& u = ts.u;
    if (u.ks > 0) {
        r.ug = host_cx<R>(u.gr, u.gi);
        r.ug16 = host_cx<R>(u.g16r, u.g16i);
        r.uc = host_cx<R>(u.cr, u.ci);
        r.uk = host_cx<R>(u.kr, u.ki);
        for (int k = 0; k < 16; k++) r.upow[k] = host_cx<R>(u.pr[k], u.pi[k]);
        r.us = (const typename V2<R>::T*)u.s;
        r.uks = u.ks;
        r.unlev = u.nlev;
    }
    return r;
}

template <typename R, int C>
static void cnx_reg_c(bool imag, dim3 grid, cudaStream_t s, const typename V2<R>::T* in, typename V2<R>::T* out,
                      const KParams& p, const Tabs<R>& t, double* partials) {
    if (imag)
        launch_pdl(k_cnx_reg<R, true, C>, grid, dim3(32), 0, s, in, out, p, t, partials);
    else
        launch_pdl(k_cnx_reg<R, false, C>, grid, dim3(32), 0, s, in, out, p, t, partials);
}

template <typename R>
static void launch_cnx_reg(int C, bool imag, dim3 grid, cudaStream_t s, const typename V2<R>::T* in,
                           typename V2<R>::T* out, const KParams& p, const Tabs<R>& t, double* partials) {
    switch (C) {
        case 1: cnx_reg_c<R, 1>(imag, grid, s, in, out, p, t, partials); break;
        case 2: cnx_reg_c<R, 2>(imag, grid, s, in, out, p, t, partials); break;
        case 4: cnx_reg_c<R, 4>(imag, grid, s, in, out, p, t, partials); break;
        case 8: cnx_reg_c<R, 8>(imag, grid, s, in, out, p, t, partials); break;
        case 16: cnx_reg_c<R, 16>(imag, grid, s, in, out, p, t, partials); break;
        default: cnx_reg_c<R, 32>(imag, grid, s, in, out, p, t, partials); break;
    }
}

template <typename R, int C>
static void cny_reg_c(bool imag, dim3 grid, cudaStream_t s, const typename V2<R>::T* in, typename V2<R>::T* out,
                      const KParams& p, const Tabs<R>& t, double* partials, DevScalars* sc, int renorm,
                      int advance) {
    if (imag)
        launch_pdl(k_cny_reg<R, true, C>, grid, dim3(32), 0, s, in, out, p, t, partials, sc, renorm, advance);
    else
        launch_pdl(k_cny_reg<R, false, C>, grid, dim3(32), 0, s, in, out, p, t, partials, sc, renorm, advance);
}

template <typename R>
static void launch_cny_reg(int C, bool imag, dim3 grid, cudaStream_t s, const typename V2<R>::T* in,
                           typename V2<R>::T* out, const KParams& p, const Tabs<R>& t, double* partials,
                           DevScalars* sc, int renorm, int advance) {
    switch (C) {
        case 1: cny_reg_c<R, 1>(imag, grid, s, in, out, p, t, partials, sc, renorm, advance); break;
        case 2: cny_reg_c<R, 2>(imag, grid, s, in, out, p, t, partials, sc, renorm, advance); break;
        case 4: cny_reg_c<R, 4>(imag, grid, s, in, out, p, t, partials, sc, renorm, advance); break;
        case 8: cny_reg_c<R, 8>(imag, grid, s, in, out, p, t, partials, sc, renorm, advance); break;
        case 16: cny_reg_c<R, 16>(imag, grid, s, in, out, p, t, partials, sc, renorm, advance); break;
        default: cny_reg_c<R, 32>(imag, grid, s, in, out, p, t, partials, sc, renorm, advance); break;
    }
}

// Allow a kernel the device's opt-in shared memory minus its static shared memory.
template <typename K> static cudaError_t allow_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (!e) e = cudaFuncGetAttributes(&fa, kernel);
    if (!e) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

template <typename R, bool IMAG, int C> static cudaError_t pwx_allow() {
    return cudaFuncSetAttribute(k_pwx<R, IMAG, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pwx_smem_bytes<R, C>());
}

template <typename R, bool IMAG> static cudaError_t pwx_allow_all() {
    cudaError_t e;
    if ((e = pwx_allow<R, IMAG, 1>())) return e;
    if ((e = pwx_allow<R, IMAG, 2>())) return e;
    if ((e = pwx_allow<R, IMAG, 4>())) return e;
    if ((e = pwx_allow<R, IMAG, 8>())) return e;
    if ((e = pwx_allow<R, IMAG, 16>())) return e;
    return pwx_allow<R, IMAG, 32>();
}

template <typename R, int C>
static void pwx_c(bool imag, int rows, cudaStream_t s, const typename V2<R>::T* A, typename V2<R>::T* B,
                  const KParams& p, const DevScalars* sc, const double* omega_tab, const Tabs<R>& t,
                  const double* partials, int m, int renorm) {
    const size_t smem = pwx_smem_bytes<R, C>();
    if (imag)
        launch_pdl(k_pwx<R, true, C>, dim3(rows), dim3(kPwxThreads), smem, s, A, B, p, sc, omega_tab, t, partials, m,
                   renorm);
    else
        launch_pdl(k_pwx<R, false, C>, dim3(rows), dim3(kPwxThreads), smem, s, A, B, p, sc, omega_tab, t, partials,
                   m, renorm);
}

template <typename R, bool IMAG, int C> static cudaError_t step1d_allow() {
    return cudaFuncSetAttribute(k_step1d<R, IMAG, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step1d_smem_bytes<R, C>(32 * C));
}

template <typename R, bool IMAG> static cudaError_t step1d_allow_all() {
    cudaError_t e;
    if ((e = step1d_allow<R, IMAG, 1>())) return e;
    if ((e = step1d_allow<R, IMAG, 2>())) return e;
    if ((e = step1d_allow<R, IMAG, 4>())) return e;
    if ((e = step1d_allow<R, IMAG, 8>())) return e;
    if ((e = step1d_allow<R, IMAG, 16>())) return e;
    return step1d_allow<R, IMAG, 32>();
}

template <typename R, int C>
static void step1d_c(bool imag, cudaStream_t s, typename V2<R>::T* A, const KParams& p, DevScalars* sc,
                     const double* omega_tab, const Tabs<R>& t, int nsteps, int renorm) {
    const size_t smem = step1d_smem_bytes<R, C>(p.nx);
    if (imag)
        k_step1d<R, true, C><<<1, kStep1dThreads, smem, s>>>(A, p, sc, omega_tab, t, nsteps, renorm);
    else
        k_step1d<R, false, C><<<1, kStep1dThreads, smem, s>>>(A, p, sc, omega_tab, t, nsteps, renorm);
}

template <typename R>
cudaError_t Launcher<R>::step1d(cudaStream_t s, bool imag, void* A, const KParams& p, DevScalars* sc,
                                const double* omega_tab, const void* const* tabs_x, int nsteps, int renorm) {
    using T = typename V2<R>::T;
    if (p.dim != 1 || p.nx > kRegMaxN) return cudaErrorInvalidValue;
    Tabs<R> t = make_tabs<R>(tabs_x);
    KParams q = p;
    fill_derived(q);
    T* a = (T*)A;
    if constexpr (std::is_same<R, double>::value) {
        // complex128: one cluster of ceil(nx/32) CTAs (the FP64 work of a point split over three threads)
        if (p.nx > kCl1dMaxN) return cudaErrorInvalidValue;
        const unsigned Q = (unsigned)ceil_div(p.nx, 32);
        const cudaError_t e = imag ? launch_cluster(k_step1d_cl<true>, Q, dim3(kCl1dThreads), 0, s, a, q, sc,
                                                    omega_tab, t, nsteps, renorm)
                                   : launch_cluster(k_step1d_cl<false>, Q, dim3(kCl1dThreads), 0, s, a, q, sc,
                                                    omega_tab, t, nsteps, renorm);
        return e ? e : cudaGetLastError();
    }
    switch (chunk_len(p.nx)) {
        case 1: step1d_c<R, 1>(imag, s, a, q, sc, omega_tab, t, nsteps, renorm); break;
        case 2: step1d_c<R, 2>(imag, s, a, q, sc, omega_tab, t, nsteps, renorm); break;
        case 4: step1d_c<R, 4>(imag, s, a, q, sc, omega_tab, t, nsteps, renorm); break;
        case 8: step1d_c<R, 8>(imag, s, a, q, sc, omega_tab, t, nsteps, renorm); break;
        case 16: step1d_c<R, 16>(imag, s, a, q, sc, omega_tab, t, nsteps, renorm); break;
        default: step1d_c<R, 32>(imag, s, a, q, sc, omega_tab, t, nsteps, renorm); break;
    }
    return cudaGetLastError();
}

template <typename R, int C> static cudaError_t socn_allow() {
    return cudaFuncSetAttribute(k_socn<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)socn_smem_bytes<R, C>());
}

template <typename R, int C>
static void socn_c(cudaStream_t s, const typename V2<R>::T* in, typename V2<R>::T* out, const SoCnLines& L,
                   const Tabs<R>& tp, const Tabs<R>& tm, const DevScalars* sc, int scale) {
    k_socn<R, C><<<L.nlines, kSoCnThreads, socn_smem_bytes<R, C>(), s>>>(in, out, L, tp, tm, sc, scale);
}

template <typename R>
cudaError_t Launcher<R>::socn(cudaStream_t s, const void* in, void* out, const SoCnLines& L, const void* const* tabs_p,
                              const void* const* tabs_m, const DevScalars* sc, int scale) {
    using T = typename V2<R>::T;
    if (L.n > kRegMaxN) return cudaErrorInvalidValue;
    const Tabs<R> tp = make_tabs<R>(tabs_p), tm = make_tabs<R>(tabs_m);
    const T* a = (const T*)in;
    T* b = (T*)out;
    switch (chunk_len(L.n)) {
        case 1: socn_c<R, 1>(s, a, b, L, tp, tm, sc, scale); break;
        case 2: socn_c<R, 2>(s, a, b, L, tp, tm, sc, scale); break;
        case 4: socn_c<R, 4>(s, a, b, L, tp, tm, sc, scale); break;
        case 8: socn_c<R, 8>(s, a, b, L, tp, tm, sc, scale); break;
        case 16: socn_c<R, 16>(s, a, b, L, tp, tm, sc, scale); break;
        default: socn_c<R, 32>(s, a, b, L, tp, tm, sc, scale); break;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::coef_skew(cudaStream_t s, void* fa, void* fg, void* fp, void* fq, int n, double are,
                                   double aim) {
    using T = typename V2<R>::T;
    const int C = chunk_len(n);
    k_coef_skew<R><<<1, 32, 0, s>>>((T*)fa, (T*)fg, (T*)fp, (T*)fq, n, C, 32 * C, are, aim);
    return cudaGetLastError();
}

template <typename R> cudaError_t Launcher<R>::setup() {
    cudaError_t e;
    if constexpr (kUniForm<R>) {
        if ((e = allow_smem(k_cn_x<R, true, true>))) return e;
        if ((e = allow_smem(k_cn_x<R, false, true>))) return e;
        if ((e = allow_smem(k_cn_y<R, true, true>))) return e;
        if ((e = allow_smem(k_cn_y<R, false, true>))) return e;
        if constexpr (std::is_same<R, float>::value) {
            if ((e = allow_smem(k_pwx_long<true, true>))) return e;
            if ((e = allow_smem(k_pwx_long<false, true>))) return e;
            if ((e = allow_smem(k_pwx_long<true, false>))) return e;
            if ((e = allow_smem(k_pwx_long<false, false>))) return e;
        }
        if ((e = allow_smem(k_cn_y_tile<R, true, 1, kTileReal>))) return e;
        if ((e = allow_smem(k_cn_y_tile<R, false, 1, kTileReal>))) return e;
        if ((e = allow_smem(k_cn_y_tile<R, true, 2, kTileReal>))) return e;
        if ((e = allow_smem(k_cn_y_tile<R, false, 2, kTileReal>))) return e;
        if ((e = allow_smem(k_cn_y_tile<R, true, 1, kTileRealShort>))) return e;
        if ((e = allow_smem(k_cn_y_tile<R, false, 1, kTileRealShort>))) return e;
        if ((e = allow_smem(k_cn_y_tile<R, true, 2, kTileRealShort>))) return e;
        if ((e = allow_smem(k_cn_y_tile<R, false, 2, kTileRealShort>))) return e;
    }
    if ((e = socn_allow<R, 16>())) return e;
    if ((e = socn_allow<R, 32>())) return e;
    if ((e = step1d_allow_all<R, true>())) return e;
    if ((e = step1d_allow_all<R, false>())) return e;
    if ((e = pwx_allow_all<R, true>())) return e;
    if ((e = pwx_allow_all<R, false>())) return e;
    if ((e = allow_smem(k_cn_x<R, true, false>))) return e;
    if ((e = allow_smem(k_cn_x<R, false, false>))) return e;
    if ((e = allow_smem(k_cn_y<R, true, false>))) return e;
    if ((e = allow_smem(k_cn_y<R, false, false>))) return e;
    return cudaSuccess;
}

template <typename R>
cudaError_t Launcher<R>::pointwise(cudaStream_t s, bool imag, const void* A, void* B, const KParams& p,
                                   const DevScalars* sc, const double* omega_tab, int mask) {
    using T = typename V2<R>::T;
    // 64-thread blocks: the FP64 form is bound by each SM's FP64 pipe, and small
    // blocks spread the points evenly over the 152 SMs (1024 blocks at 256^2).
    dim3 block(32, p.dim == 2 ? 2 : 1);
    dim3 grid(ceil_div(p.nx, 32), p.dim == 2 ? ceil_div(p.ny, 2) : 1);
    KParams q = p;
    fill_derived(q);
    if constexpr (std::is_same<R, float>::value) {
        // complex64, even rows: two points a thread, 16-byte loads and stores (16-byte aligned:
        // every buffer starts 16-byte aligned and every row has an even number of points)
        if (p.nx % 2 == 0) {
            // 32 x 8 threads (64 x 8 points): the y neighbours of most rows are
            // loaded by the block itself (L1 hits; measured faster than 32 x 2 and 32 x 4)
            const dim3 block2(32, p.dim == 2 ? 8 : 1);
            const dim3 grid2(ceil_div(p.nx, 64), p.dim == 2 ? ceil_div(p.ny, 8) : 1);
            // the full step of a 2D grid with SO as its own instantiation (no runtime case tests)
            const bool std2d = mask == 7 && p.dim == 2 && q.so_case == 4;
            auto go = [&](auto kern) {
                launch_pdl(kern, grid2, block2, 0, s, (const float2*)A, (float2*)B, q, sc, omega_tab, mask);
            };
            if (std2d)
                imag ? go(k_pointwise2<true, true>) : go(k_pointwise2<false, true>);
            else
                imag ? go(k_pointwise2<true, false>) : go(k_pointwise2<false, false>);
            return cudaGetLastError();
        }
    }
    if (imag)
        launch_pdl(k_pointwise<R, true>, grid, block, 0, s, (const T*)A, (T*)B, q, sc, omega_tab, mask);
    else
        launch_pdl(k_pointwise<R, false>, grid, block, 0, s, (const T*)A, (T*)B, q, sc, omega_tab, mask);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::pwx(cudaStream_t s, bool imag, const void* A, void* B, const KParams& p,
                             const DevScalars* sc, const double* omega_tab, const void* const* tabs_x,
                             const double* partials, int m, int renorm) {
    using T = typename V2<R>::T;
    if (p.dim != 2 || p.nx > kRegMaxN) return cudaErrorInvalidValue;
    Tabs<R> t = make_tabs<R>(tabs_x);
    const T* a = (const T*)A;
    T* b = (T*)B;
    KParams q = p;
    fill_derived(q);
    switch (chunk_len(p.nx)) {
        case 1: pwx_c<R, 1>(imag, p.ny, s, a, b, q, sc, omega_tab, t, partials, m, renorm); break;
        case 2: pwx_c<R, 2>(imag, p.ny, s, a, b, q, sc, omega_tab, t, partials, m, renorm); break;
        case 4: pwx_c<R, 4>(imag, p.ny, s, a, b, q, sc, omega_tab, t, partials, m, renorm); break;
        case 8: pwx_c<R, 8>(imag, p.ny, s, a, b, q, sc, omega_tab, t, partials, m, renorm); break;
        case 16: pwx_c<R, 16>(imag, p.ny, s, a, b, q, sc, omega_tab, t, partials, m, renorm); break;
        default: pwx_c<R, 32>(imag, p.ny, s, a, b, q, sc, omega_tab, t, partials, m, renorm); break;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::pwx_long(cudaStream_t s, bool imag, const void* A, void* B, const KParams& p,
                                  const DevScalars* sc, const double* omega_tab, const TabSet& tabs_x, int mask,
                                  const double* partials, int m, int renorm) {
    if constexpr (!std::is_same<R, float>::value) {
        return cudaErrorNotSupported;
    } else {
        const int nwl = long_warps(p.nx);
        if (p.dim != 2 || p.nx % 2 || nwl > kPwxLongMaxGroupWarps || tabs_x.u.ks <= 0)
            return cudaErrorInvalidValue;
        const Tabs<float> t = make_tabs<float>(tabs_x);
        KParams q = p;
        fill_derived(q);
        const size_t smem = (size_t)3 * 32 * nwl * kLongS * sizeof(cx<float>);
        const bool std2d = mask == 7 && q.so_case == 4;
        auto go = [&](auto kern) {
            launch_pdl(kern, dim3(p.ny), dim3(96 * nwl), smem, s, (const float2*)A, (float2*)B, q, sc, omega_tab, t,
                       mask, partials, m, renorm);
        };
        if (std2d)
            imag ? go(k_pwx_long<true, true>) : go(k_pwx_long<false, true>);
        else
            imag ? go(k_pwx_long<true, false>) : go(k_pwx_long<false, false>);
        return cudaGetLastError();
    }
}

template <typename R>
cudaError_t Launcher<R>::cn_x(cudaStream_t s, bool imag, bool last, const void* in, void* out, const KParams& p,
                              const TabSet& tabs, const Geometry& g, double* partials, DevScalars* sc,
                              int renorm, int advance) {
    using T = typename V2<R>::T;
    Tabs<R> t = make_tabs<R>(tabs);
    if (g.reg_x && !(kUniForm<R> && x_tiled(g, tabs))) {
        launch_cnx_reg<R>(chunk_len(p.nx), imag, dim3(g.blocks_x), s, (const T*)in, (T*)out, p, t,
                          last ? partials : nullptr);
        return cudaGetLastError();
    }
    const dim3 block(32 * g.wx), grid(g.blocks_x);
    double* part = last ? partials : nullptr;
    auto go = [&](auto kern) { launch_pdl(kern, grid, block, g.smem_x, s, (const T*)in, (T*)out, p, t, part); };
    if (kUniForm<R> && t.uks > 0) {
        if constexpr (kUniForm<R>) imag ? go(k_cn_x<R, true, true>) : go(k_cn_x<R, false, true>);
    } else {
        imag ? go(k_cn_x<R, true, false>) : go(k_cn_x<R, false, false>);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::cn_y(cudaStream_t s, bool imag, const void* in, void* out, const KParams& p,
                              const TabSet& tabs, const Geometry& g, double* partials, DevScalars* sc,
                              int renorm, int advance, int finalize, bool head_scale) {
    using T = typename V2<R>::T;
    Tabs<R> t = make_tabs<R>(tabs);
    double* part = finalize ? partials : nullptr;
    if (y_tiled(g, tabs, in, out)) {
        if constexpr (kUniForm<R>) {
            const int hc = tabs.u.hc, rtc = g.tile_rt;
            const dim3 tb(32 * (rtc + 2 * hc)), tg(g.blocks_yt);
            const size_t sm = (size_t)(rtc + 2 * hc) * kLongC * 32 * sizeof(cx<R>);
            DevScalars* hs = head_scale ? sc : nullptr;
            auto go = [&](auto kern) {
                launch_pdl(kern, tg, tb, sm, s, (const T*)in, (T*)out, p, t, part, hs, renorm, advance);
            };
            if (rtc == kTileReal) {
                if (hc == 1)
                    imag ? go(k_cn_y_tile<R, true, 1, kTileReal>) : go(k_cn_y_tile<R, false, 1, kTileReal>);
                else
                    imag ? go(k_cn_y_tile<R, true, 2, kTileReal>) : go(k_cn_y_tile<R, false, 2, kTileReal>);
            } else {
                if (hc == 1)
                    imag ? go(k_cn_y_tile<R, true, 1, kTileRealShort>) : go(k_cn_y_tile<R, false, 1, kTileRealShort>);
                else
                    imag ? go(k_cn_y_tile<R, true, 2, kTileRealShort>) : go(k_cn_y_tile<R, false, 2, kTileRealShort>);
            }
            return cudaGetLastError();
        }
    }
    if (g.reg_y) {
        launch_cny_reg<R>(chunk_len(p.ny), imag, dim3(g.blocks_y), s, (const T*)in, (T*)out, p, t,
                          finalize ? partials : nullptr, head_scale ? sc : nullptr, renorm, advance);
        return cudaGetLastError();
    }
    // tiles of 1, 2 or 4 columns within the block limit (the kernel splits its staging
    // index by shift and mask)
    if ((g.wy & (g.wy - 1)) || g.wy > 4 || g.wy * long_warps(p.ny) > kLongMaxWarps) return cudaErrorInvalidValue;
    const dim3 block(32 * g.wy * long_warps(p.ny)), grid(g.blocks_y);
    const bool uni = kUniForm<R> && t.uks > 0;
    auto go = [&](auto kern) { kern<<<grid, block, g.smem_y, s>>>((const T*)in, (T*)out, p, t, g.wy, part); };
    if (uni) {
        if constexpr (kUniForm<R>) imag ? go(k_cn_y<R, true, true>) : go(k_cn_y<R, false, true>);
    } else {
        imag ? go(k_cn_y<R, true, false>) : go(k_cn_y<R, false, false>);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::coef(cudaStream_t s, void* fa, void* fg, void* fp, void* fq, int n, double bre, double bim) {
    using T = typename V2<R>::T;
    k_coef<R><<<1, 32, 0, s>>>((T*)fa, (T*)fg, (T*)fp, (T*)fq, n, chunk_len(n), table_len(n), n > kRegMaxN ? 1 : 0,
                               bre, bim);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::uni(cudaStream_t s, int n, double bre, double bim, void* s_dev, UniHost* u) {
    using C = std::complex<double>;
    *u = UniHost{};
    const C b(bre, bim), d = 1.0 + 2.0 * b;
    // the pivot limit: the root of u^2 - d u + b^2 with |u| > |b|, polished by the
    // contraction u <- d - b^2 / u itself
    const C disc = std::sqrt(d * d - 4.0 * b * b);
    C piv = (d + disc) * 0.5, alt = (d - disc) * 0.5;
    if (std::abs(alt) > std::abs(piv)) piv = alt;
    for (int k = 0; k < 8; k++) piv = d - b * b / piv;
    const C a = 1.0 / piv, g = b / piv;
    if (!kUniForm<R> || !(std::abs(g) < 1.0)) return cudaSuccess;
    C g16 = g;
    for (int k = 0; k < 4; k++) g16 = g16 * g16;
    // s = T'^{-1} e_0: forward z_0 = 1, z_i = g z_{i-1}; backward q_{n-1} = z_{n-1},
    // q_i = z_i + g q_{i+1}; s = a q
    std::vector<C> z(n), q(n);
    z[0] = 1.0;
    for (int i = 1; i < n; i++) z[i] = g * z[i - 1];
    q[n - 1] = z[n - 1];
    for (int i = n - 2; i >= 0; i--) q[i] = z[i] + g * q[i + 1];
    const C delta = d - piv;
    const C s0 = a * q[0];
    const C c = delta / (1.0 + delta * s0);
    const double cut = std::ldexp(1.0, -64);
    int ks = 0;
    for (int i = 0; i < n; i++)
        if (std::abs(c * a * q[i]) >= cut) ks = i + 1;
    if (ks > kUniMaxS) return cudaSuccess;
    ks = std::max(ks, 1);
    int nlev = 0;
    for (double f = std::abs(g16); nlev < 5 && !(f < cut); f *= f) nlev++;
    // the sweep's result from q = w / a: 2 a q - x, or x + 2 bt a q (increment form, complex64)
    const C k = is_f32<R>() ? 2.0 * b * a : 2.0 * a;
    using T = typename V2<R>::T;
    std::vector<T> hs(ks);
    for (int i = 0; i < ks; i++) {
        const C si = a * q[i];
        hs[i] = host_elem<R>(si.real(), si.imag());
    }
    // (s_dev null: the host figures only, nothing copied)
    if (s_dev) {
        cudaError_t e = cudaMemcpyAsync(s_dev, hs.data(), sizeof(T) * ks, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns; keep the
    // stream order with the kernels that read s
    *u = UniHost{};
    u->gr = g.real();
    u->gi = g.imag();
    u->g16r = g16.real();
    u->g16i = g16.imag();
    u->cr = c.real();
    u->ci = c.imag();
    u->kr = k.real();
    u->ki = k.imag();
    C pw = 1.0;
    for (int j = 0; j < 16; j++) {
        pw *= g;
        u->pr[j] = pw.real();
        u->pi[j] = bim == 0.0 ? pw.real() : pw.imag();
    }
    u->ks = ks;
    u->nlev = nlev;
    // the row-tiled y sweep: hc halo chunks, the first with |g^16|^hc below 2^-64
    // (the weight of the nearest chunk left out), and the start correction
    // within the top tile
    {
        int hc = 1;
        for (double f = std::abs(g16); hc <= kTileMaxHalo && !(f < cut); f *= std::abs(g16)) hc++;
        u->hc = (hc <= kTileMaxHalo && ks <= kTileRows) ? hc : 0;
    }
    u->s = s_dev;
    return cudaSuccess;
}

template <typename R> cudaError_t Launcher<R>::flush(cudaStream_t s, void* A, size_t plane, const DevScalars* sc) {
    using T = typename V2<R>::T;
    size_t total = 3 * plane;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4 * kNormBlocks) blocks = 4 * kNormBlocks;
    k_flush<R><<<blocks, 256, 0, s>>>((T*)A, plane, sc);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::norms(cudaStream_t s, const void* A, size_t plane, double cell, int renorm, double mag,
                               double* partials, DevScalars* sc, int advance) {
    using T = typename V2<R>::T;
    k_norms<R><<<kNormBlocks, 256, 0, s>>>((const T*)A, plane, cell, renorm, mag, partials, sc, advance);
    return cudaGetLastError();
}

template <typename R>
cudaError_t Launcher<R>::observables(cudaStream_t s, const void* A, const KParams& p, double omega_t,
                                     double* partials, DevScalars* sc) {
    using T = typename V2<R>::T;
    dim3 block(32, 4);
    dim3 grid(ceil_div(p.nx, 32), ceil_div(p.ny, 4));
    k_observables<R><<<grid, block, 0, s>>>((const T*)A, p, omega_t, partials, sc);
    return cudaGetLastError();
}

}  // namespace sgpe
