// sgpe_socn.cuh -- the SO substep by Crank-Nicolson (the unitary variant of
// the explicit-Euler SO substep of Appendix A Eqs. (p1)-(p2)).
//
// Along one grid line the SO operator of Sec. 2 is H = g S p, p = -i D (D the
// central first difference with zero ghosts, spacing h), S one of the spin-1
// matrices Sigma_x, Sigma_y, Sigma_z of Eq. (smat) and g a real strength (1D:
// gamma; 2D x lines: -gamma with S = Sigma_y; 2D y lines: eta gamma with S =
// Sigma_x). Crank-Nicolson: (I + z/2 H) psi' = (I - z/2 H) psi. S has the
// eigenvalues +1, 0, -1 with eigenvectors u_k (the columns of U, fixed 3x3),
// so in the rotated components phi = U^H psi the system splits into three
// scalar lines: phi_0 is unchanged, and phi_(+-1) solve
//   T phi' = (2 I - T) phi,  T = I + a_m (S+ - S-),  a_m = -i z g m / (4 h),
// a tridiagonal matrix with opposite off-diagonals (S+-: shift by one point).
// Each line is solved in increment form, phi' = phi + 2 e with
// T e = -a_m (phi_(i+1) - phi_(i-1)), by the lane-chunk scan of the kinetic
// sweeps with skew tables (k_coef_skew). The result is psi' = U phi'.
//
// One block of three warps per line (n <= 1024 points): the line's three
// components are loaded, rotated and staged in shared memory in the lanes'
// padded chunk layout; warps 0 and 2 solve phi_(+1) and phi_(-1); all threads
// rotate back and store.
#pragma once
#include "sgpe_cn.cuh"

namespace sgpe {

// One family of lines of one grid (x lines or y lines) for the SO-CN substep.
struct SoCnLines {
    double ur[9], ui[9];      // U[j][k] = ur[3j + k] + i ui[3j + k]: component j of the eigenvector of m_k
    double are, aim;          // a of m = +1 (m = -1 takes -a)
    int n, nlines;            // points per line, lines
    long long stride, lstride;  // element distance between the points of a line, between lines
    long long plane;          // elements per spin component
};

constexpr int kSoCnThreads = 96;

// One product term u v (or conj(u) v) of the eigenbasis rotation. For the FP32
// state the rounding remainder ul of each entry of U (1/sqrt2 is not an FP32
// number) is added inside the fused multiply-adds, before the product is first
// rounded: each term is then rounded once from a value accurate to ~1e-15. Added
// after the rounded product the remainder would be lost, and the rounding of
// 1/sqrt2 would shrink the norm by ~1.3e-8 per rotation, four rotations a step.
template <bool CONJ, typename R>
__device__ __forceinline__ cx<R> rot_term(cx<R> u, cx<R> ul, cx<R> v) {
    if constexpr (is_f32<R>()) {
        const cx<R> c = CONJ ? cmul(ul, v) : mul(ul, v);
        if (CONJ)
            return {fma(u.re, v.re, fma(u.im, v.im, c.re)), fma(u.re, v.im, fma(-u.im, v.re, c.im))};
        return {fma(u.re, v.re, fma(-u.im, v.im, c.re)), fma(u.re, v.im, fma(u.im, v.re, c.im))};
    } else {
        return CONJ ? cmul(u, v) : mul(u, v);
    }
}

template <typename R, int C> constexpr size_t socn_smem_bytes() {
    return (size_t)3 * 32 * (C + 1) * sizeof(typename V2<R>::T);
}

// COEF of the skew matrix T = tridiag(-a, 1, a) of n points for one m:
// u_0 = 1, u_i = 1 + a^2 / u_(i-1); forward y_i = fa_i x_i + fg_i y_(i-1) with
// fa = 1/u, fg = a/u; backward w_i = y_i - fg_i w_(i+1). fp: chunk prefix
// products of fg, fq: chunk suffix products of -fg. Tables padded with zeros
// to len = 32 C entries. One thread; FP64, stored rounded to R.
template <typename R>
__global__ void k_coef_skew(typename V2<R>::T* fa, typename V2<R>::T* fg, typename V2<R>::T* fp,
                            typename V2<R>::T* fq, int n, int C, int len, double are, double aim) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const cx<R> zero = {R(0), R(0)};
    for (int i = n; i < len; i++) {
        st<R>(fa, i, zero);
        st<R>(fg, i, zero);
    }
    const double a2r = are * are - aim * aim, a2i = 2.0 * are * aim;
    double ur = 1.0, ui = 0.0;
    for (int i = 0; i < n; i++) {
        if (i > 0) {
            double qr, qi;
            cdiv(a2r, a2i, ur, ui, &qr, &qi);
            ur = 1.0 + qr;
            ui = qi;
        }
        double xr, xi, gr, gi;
        cdiv(1.0, 0.0, ur, ui, &xr, &xi);
        cdiv(are, aim, ur, ui, &gr, &gi);
        st<R>(fa, i, cx<R>{to_r<R>(xr), to_r<R>(xi)});
        st<R>(fg, i, cx<R>{to_r<R>(gr), to_r<R>(gi)});
    }
    for (int k0 = 0; k0 < len; k0 += C) {
        const int k1 = k0 + C;
        double Pr = 1.0, Pi = 0.0;
        for (int i = k0; i < k1; i++) {
            const cx<R> g = unpack(fg[i]);
            const double gr = dbl(g.re), gi = dbl(g.im);
            const double tr = Pr * gr - Pi * gi, ti = Pr * gi + Pi * gr;
            Pr = tr;
            Pi = ti;
            st<R>(fp, i, cx<R>{to_r<R>(Pr), to_r<R>(Pi)});
        }
        Pr = 1.0;
        Pi = 0.0;
        for (int i = k1 - 1; i >= k0; i--) {
            const cx<R> g = unpack(fg[i]);
            const double gr = -dbl(g.re), gi = -dbl(g.im);
            const double tr = Pr * gr - Pi * gi, ti = Pr * gi + Pi * gr;
            Pr = tr;
            Pi = ti;
            st<R>(fq, i, cx<R>{to_r<R>(Pr), to_r<R>(Pi)});
        }
    }
}

// The SO-CN substep on one family of lines: in -> out (may be the same buffer).
// scale: apply the pending renormalisation scale of sc on load (the first
// kernel of a step). tp, tm: the skew tables of m = +1 and m = -1.
template <typename R, int C>
__global__ void __launch_bounds__(kSoCnThreads) k_socn(const typename V2<R>::T* in, typename V2<R>::T* out,
                                                      SoCnLines L, Tabs<R> tp, Tabs<R> tm,
                                                      const DevScalars* __restrict__ sc, int scale) {
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char socn_smem[];
    T* row = reinterpret_cast<T*>(socn_smem);
    constexpr int S = 32 * (C + 1);
    const int n = L.n;
    const size_t base = (size_t)blockIdx.x * (size_t)L.lstride;
    const size_t plane = (size_t)L.plane, stride = (size_t)L.stride;
    const cx<R> zero = {R(0), R(0)};
    pdl_wait();
    R ds[3];
#pragma unroll
    for (int j = 0; j < 3; j++) ds[j] = scale ? scale_of<R>(sc, j) : R(1);
    // U and, for the FP32 state, the rest of each entry after rounding to FP32 (Ul, see rot_term)
    cx<R> U[9], Ul[9];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        U[q] = {to_r<R>(L.ur[q]), to_r<R>(L.ui[q])};
        Ul[q] = is_f32<R>() ? cx<R>{to_r<R>(L.ur[q] - dbl(U[q].re)), to_r<R>(L.ui[q] - dbl(U[q].im))} : zero;
    }
    for (int i = threadIdx.x; i < 32 * C; i += kSoCnThreads) {
        cx<R> v[3];
#pragma unroll
        for (int j = 0; j < 3; j++) v[j] = i < n ? scl(ds[j], ldc<R>(in, j * plane + base + (size_t)i * stride)) : zero;
        const int slot = (i / C) * (C + 1) + (i % C);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            // phi_k = sum_j conj(U[j][k]) psi_j
            cx<R> ph = rot_term<true>(U[k], Ul[k], v[0]);
            ph = add(ph, rot_term<true>(U[3 + k], Ul[3 + k], v[1]));
            ph = add(ph, rot_term<true>(U[6 + k], Ul[6 + k], v[2]));
            row[k * S + slot] = pack(ph);
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp != 1) {
        const Tabs<R>& t = warp == 0 ? tp : tm;
        const R sg = warp == 0 ? R(1) : R(-1);
        const cx<R> a = {sg * to_r<R>(L.are), sg * to_r<R>(L.aim)};
        T* r = row + warp * S;
        const int i0 = lane * C;
        cx<R> x[C], e[C];
#pragma unroll
        for (int m = 0; m < C; m++) x[m] = unpack(r[lane * (C + 1) + m]);
        // e_i = -a (x_(i+1) - x_(i-1)); points past n hold zeros
        cx<R> prev = shup(x[C - 1], 1), last = shdn(x[0], 1);
        if (lane == 0) prev = zero;
        if (lane == 31) last = zero;
#pragma unroll
        for (int m = 0; m < C; m++) {
            const cx<R> nxt = (m + 1 < C) ? x[m + 1] : last;
            const cx<R> d = sub(nxt, prev);
            e[m] = {-(a.re * d.re - a.im * d.im), -(a.re * d.im + a.im * d.re)};
            prev = x[m];
        }
        LaneTabs<R, false, C> lt;
        lt.init(t, i0);
        solve_chunk<R, false, C, true>(e, lt);
#pragma unroll
        for (int m = 0; m < C; m++) {
            const cx<R> o = {fma(R(2), e[m].re, x[m].re), fma(R(2), e[m].im, x[m].im)};
            r[lane * (C + 1) + m] = pack(o);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kSoCnThreads) {
        const int slot = (i / C) * (C + 1) + (i % C);
        const cx<R> p0 = unpack(row[slot]), p1 = unpack(row[S + slot]), p2 = unpack(row[2 * S + slot]);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            // psi_j = sum_k U[j][k] phi_k
            cx<R> o = rot_term<false>(U[3 * j], Ul[3 * j], p0);
            o = add(o, rot_term<false>(U[3 * j + 1], Ul[3 * j + 1], p1));
            o = add(o, rot_term<false>(U[3 * j + 2], Ul[3 * j + 2], p2));
            st<R>(out, j * plane + base + (size_t)i * stride, o);
        }
    }
}

}  // namespace sgpe
