// sgpe_step1d_cl.cuh -- the complex128 1D step loop in one thread-block
// cluster (lines of at most 256 points, all nsteps steps in one launch).
//
// Why: a 1D grid is far too small to fill the GPU, so its step is bound by the
// length of each thread's dependent FP64 chain: on GB300 one warp's FP64
// instruction holds its SM sub-partition for about 64 cycles, so a thread
// that runs all pointwise substeps of a point (~160 FP64 instructions) needs
// ~5 us per step however many SMs are used. Here the work of a point is split
// over three threads (warp j of each CTA takes spin component j) and the state
// stays in the cluster's shared memory for all steps:
//   * CTA q of the cluster (Q = ceil(nx/32) CTAs, 1..8) holds points
//     [32q, 32q + 32) of the three lines; lane l of warp j owns point 32q + l
//     of component j.
//   * Pointwise substeps (Sec. 3 SO, CALCNU, HERM): each thread computes the
//     update of its own component; the values of the other two components at
//     the same point come from shared memory after each substep. The edge
//     neighbours of the SO stencil come from the adjacent CTAs' shared memory.
//   * CN along x (Sec. 3 LU): one point per lane; the chunk maps of the
//     forward and backward recurrences (with the precomputed LU factors fa, fg)
//     are composed by shuffles inside each warp and then across the cluster's
//     CTAs through distributed shared memory; both compositions stop once the
//     composed factor is negligible (see tiny_carry).
//   * Renormalisation (Eq. (DJ2) / (DJ)): each warp's FP64 norm partial goes
//     to every CTA; every CTA sums the Q partials of each component in the
//     same order and forms the same scale, applied at the next step's first
//     load, as on the other paths.
// Three cluster barriers per step order the exchanges; the kernel has no
// spin-waits and no early returns (every thread reaches every barrier).
#pragma once
#include "sgpe_cn.cuh"
#include "sgpe_launch.h"

namespace sgpe {

constexpr int kCl1dMaxQ = kCl1dMaxN / 32;  // CTAs per cluster (8: the portable maximum)
constexpr int kCl1dThreads = 96;           // warp j = spin component j

__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Cluster barrier, executed uniformly by every thread of every CTA (__syncwarp
// first: the .aligned forms want the warp converged). The release arrive
// publishes this thread's earlier shared-memory stores (own or a peer's) to the
// threads that pass the acquire wait; it is also a barrier of the CTA.
__device__ __forceinline__ void cl_sync() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Generic address of the same shared-memory object in CTA `rank` of the cluster.
template <typename T> __device__ __forceinline__ T* cl_map(T* p, unsigned rank) {
    uint64_t r;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"((uint64_t)p), "r"(rank));
    return reinterpret_cast<T*>(r);
}

// SO update of component j alone (the formulas of so_point for the 1D cases):
// h_j from the raw differences X of the three components, u_j -= z h_j.
template <bool IMAG>
__device__ __forceinline__ cx<double> so_comp(int j, cx<double> u, const cx<double> (&X)[3],
                                              const double (&gx)[3], int so_case) {
    cx<double> h = {0.0, 0.0};
    if (so_case == 1) {
        if (j != 1)
            h = {gx[1] * X[1].im, -gx[1] * X[1].re};
        else
            h = {fma(gx[0], X[0].im, gx[2] * X[2].im), -fma(gx[0], X[0].re, gx[2] * X[2].re)};
    } else if (so_case == 2) {
        const cx<double> hm = scl(gx[1], X[1]);
        if (j == 0)
            h = {-hm.re, -hm.im};
        else if (j == 2)
            h = hm;
        else
            h = {fma(gx[0], X[0].re, -gx[2] * X[2].re), fma(gx[0], X[0].im, -gx[2] * X[2].im)};
    } else if (so_case == 3) {
        if (j == 0)
            h = {gx[0] * X[0].im, -gx[0] * X[0].re};
        else if (j == 2)
            h = {-gx[2] * X[2].im, gx[2] * X[2].re};
        else
            return u;
    } else {
        return u;
    }
    return sub(u, zunit<IMAG>(h));
}

// CALCNU factor of component j (the exponent of calcnu_point_dt) applied to u.
template <bool IMAG>
__device__ __forceinline__ cx<double> calcnu_comp(int j, cx<double> u, const cx<double> (&w)[3], double Vn,
                                                  const KParams& p) {
    const double rp = nrm(w[0]), r0 = nrm(w[1]), rm = nrm(w[2]);
    const double base = fma(p.kd[KC_NC0], rp + r0 + rm, Vn);
    const double nc2 = p.kd[KC_NC2];
    const double x = j == 0 ? fma(nc2, rp - rm + r0, base) : j == 1 ? fma(nc2, rp + rm, base)
                                                                    : fma(nc2, rm - rp + r0, base);
    if (IMAG) return scl(exp_small(x), u);
    double s, c;
    sincos_small(x, &s, &c);
    return mul(cx<double>{c, s}, u);
}

// HERM update of component j (the formulas of herm_point for that component).
template <bool IMAG>
__device__ __forceinline__ cx<double> herm_comp(int j, const cx<double> (&u)[3], double c2, double Ot,
                                                const KParams& p) {
    cx<double> a = cmul(u[2], u[1]);  // psi_-^* psi_0
    a = {fma(c2, a.re, Ot), c2 * a.im};
    cx<double> b = cmul(u[1], u[0]);  // psi_0^* psi_+
    b = {fma(c2, b.re, Ot), c2 * b.im};
    const double na = nrm(a), nb = nrm(b);
    const double C2 = na + nb;
    double s, k;
    herm_coeffs_dt<IMAG>(C2, p, &s, &k);
    if (j == 0) {
        const cx<double> Ap = mul(a, u[1]);
        const cx<double> Bp = axpy(na, u[0], mul(mul(a, b), u[2]));
        return axpy(k, Bp, axpy(-s, zunit<IMAG>(Ap), u[0]));
    }
    if (j == 1) {
        const cx<double> A0 = add(cmul(a, u[0]), mul(b, u[2]));
        const cx<double> B0 = scl(C2, u[1]);
        return axpy(k, B0, axpy(-s, zunit<IMAG>(A0), u[1]));
    }
    const cx<double> Am = cmul(b, u[1]);
    const cx<double> Bm = axpy(nb, u[2], cmul(mul(a, b), u[0]));
    return axpy(k, Bm, axpy(-s, zunit<IMAG>(Am), u[2]));
}

struct Cl1dShared {
    double2 st[3][32];            // the CTA's slice of the three lines (raw state)
    double2 xX[3][32];            // SO: raw differences of each component
    double2 xa[3][32], xb[3][32];  // values after SO (for CALCNU) and after CALCNU (for HERM)
    double2 fA[3][kCl1dMaxQ], fB[3][kCl1dMaxQ];  // forward segment maps of the cluster's CTAs
    double2 bA[3][kCl1dMaxQ], bB[3][kCl1dMaxQ];  // backward segment maps
    double part[3][kCl1dMaxQ];                   // norm partials of the cluster's CTAs
    double ds[3];
};

// Launched as one cluster of Q = ceil(nx/32) CTAs of kCl1dThreads threads
// (grid Q, cluster Q), nx <= kCl1dMaxN. A: the state [3][nx]; t: the x tables
// of the step's mode (fa, fg used; entries past nx are zero).
template <bool IMAG>
__global__ void __launch_bounds__(kCl1dThreads, 1)
    k_step1d_cl(double2* __restrict__ A, KParams p, DevScalars* sc, const double* __restrict__ omega_tab,
                Tabs<double> t, int nsteps, int renorm) {
    __shared__ Cl1dShared S;
    const unsigned q = cl_rank();
    const unsigned Q = gridDim.x;
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = p.nx;
    const int i = (int)q * 32 + lane;
    const bool valid = i < nx;
    const cx<double> zero = {0.0, 0.0};
    S.st[j][lane] = valid ? __ldcg(A + (size_t)j * nx + i) : make_double2(0.0, 0.0);
    if (threadIdx.x < 3) S.ds[threadIdx.x] = sc->scale[threadIdx.x];
    const int step0 = sc->step_idx;
    const cx<double> fa = valid ? tld<double>(t.fa, i) : zero;
    const cx<double> fg = valid ? tld<double>(t.fg, i) : zero;
    const int kx = i - nx / 2;
    const double Vn = p.kd[KC_NVX] * double(kx * kx);
    const double c2 = p.kd[KC_C2];
    double dlast[3] = {S.ds[0], S.ds[1], S.ds[2]};
    bool finite = true;
    __syncthreads();
    cl_sync();  // every CTA has loaded its slice: neighbours may be read
    for (int s = 0; s < nsteps; s++) {
        const double Ot = omega_tab ? __ldg(omega_tab + step0 + s) * 0.70710678118654752440 : p.kd[KC_OMEGA];
        // --- pointwise substeps of (point i, component j)
        const cx<double> raw = unpack(S.st[j][lane]);
        const cx<double> left = lane > 0 ? unpack(S.st[j][lane - 1])
                                         : (q > 0 ? unpack(*cl_map(&S.st[j][31], q - 1)) : zero);
        const cx<double> right = lane < 31 ? unpack(S.st[j][lane + 1])
                                           : (q + 1 < Q ? unpack(*cl_map(&S.st[j][0], q + 1)) : zero);
        const double d[3] = {S.ds[0], S.ds[1], S.ds[2]};
        cx<double> u = scl(d[j], raw);
        if (p.so_case) {
            S.xX[j][lane] = pack(sub(right, left));
            __syncthreads();
            const cx<double> X[3] = {unpack(S.xX[0][lane]), unpack(S.xX[1][lane]), unpack(S.xX[2][lane])};
            double gx[3];
            if (p.renorm != 2) {
                gx[0] = gx[1] = gx[2] = p.kd[KC_HX] * d[0];
            } else {
#pragma unroll
                for (int k = 0; k < 3; k++) gx[k] = p.kd[KC_HX] * d[k];
            }
            u = so_comp<IMAG>(j, u, X, gx, p.so_case);
        }
        S.xa[j][lane] = pack(u);
        __syncthreads();
        {
            const cx<double> w[3] = {unpack(S.xa[0][lane]), unpack(S.xa[1][lane]), unpack(S.xa[2][lane])};
            u = calcnu_comp<IMAG>(j, u, w, Vn, p);
        }
        S.xb[j][lane] = pack(u);
        __syncthreads();
        {
            const cx<double> w[3] = {unpack(S.xb[0][lane]), unpack(S.xb[1][lane]), unpack(S.xb[2][lane])};
            u = herm_comp<IMAG>(j, w, c2, Ot, p);
        }
        const cx<double> x = valid ? u : zero;  // the CN right-hand side
        // --- CN along x, forward: y_i = fa_i x_i + fg_i y_{i-1}
        const cx<double> yl = tmul<IMAG>(fa, x);
        cx<double> sA = fg, sB = yl;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const cx<double> Ap = shup(sA, off), Bp = shup(sB, off);
            if (lane >= off) {
                sB = tfma<IMAG>(sA, Bp, sB);
                sA = tmul<IMAG>(sA, Ap);
            }
            if (scan_done(lane < 2 * off, sA)) break;
        }
        if (lane == 31)
            for (unsigned r = 0; r < Q; r++) {
                *cl_map(&S.fA[j][q], r) = pack(sA);
                *cl_map(&S.fB[j][q], r) = pack(sB);
            }
        cl_sync();
        // y at the last point of the previous CTAs' segments
        cx<double> cinC = zero;
        if (q > 0) {
            cinC = unpack(S.fB[j][q - 1]);
            cx<double> w = unpack(S.fA[j][q - 1]);
            for (int r = (int)q - 2; r >= 0; r--) {
                if (tiny_carry(w.re) && tiny_carry(w.im)) break;
                cinC = tfma<IMAG>(w, unpack(S.fB[j][r]), cinC);
                w = tmul<IMAG>(w, unpack(S.fA[j][r]));
            }
        }
        const cx<double> Au = shup(sA, 1), Bu = shup(sB, 1);
        const cx<double> yprev = lane == 0 ? cinC : tfma<IMAG>(Au, cinC, Bu);
        const cx<double> y = tfma<IMAG>(fg, yprev, yl);
        // --- backward: w_i = y_i + fg_i w_{i+1}
        sA = fg;
        sB = y;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const cx<double> An = shdn(sA, off), Bn = shdn(sB, off);
            if (lane + off < 32) {
                sB = tfma<IMAG>(sA, Bn, sB);
                sA = tmul<IMAG>(sA, An);
            }
            if (scan_done(lane + 2 * off >= 32, sA)) break;
        }
        if (lane == 0)
            for (unsigned r = 0; r < Q; r++) {
                *cl_map(&S.bA[j][q], r) = pack(sA);
                *cl_map(&S.bB[j][q], r) = pack(sB);
            }
        cl_sync();
        cx<double> cbC = zero;
        if (q + 1 < Q) {
            cbC = unpack(S.bB[j][q + 1]);
            cx<double> w = unpack(S.bA[j][q + 1]);
            for (unsigned r = q + 2; r < Q; r++) {
                if (tiny_carry(w.re) && tiny_carry(w.im)) break;
                cbC = tfma<IMAG>(w, unpack(S.bB[j][r]), cbC);
                w = tmul<IMAG>(w, unpack(S.bA[j][r]));
            }
        }
        const cx<double> An = shdn(sA, 1), Bn = shdn(sB, 1);
        const cx<double> wnext = lane == 31 ? cbC : tfma<IMAG>(An, cbC, Bn);
        const cx<double> wv = tfma<IMAG>(fg, wnext, y);
        const cx<double> o = valid ? cx<double>{fma(2.0, wv.re, -x.re), fma(2.0, wv.im, -x.im)} : zero;
        S.st[j][lane] = pack(o);
        // --- norm partials to every CTA, then the same scale everywhere
        const double pn = warp_sum(nrm(o));
        if (lane == 0)
            for (unsigned r = 0; r < Q; r++) *cl_map(&S.part[j][q], r) = pn;
        cl_sync();
        if (threadIdx.x == 0) {
            double N[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (unsigned r = 0; r < Q; r++) acc += S.part[k][r];
                N[k] = acc * p.cell;
            }
            const bool fin = isfinite(N[0]) && isfinite(N[1]) && isfinite(N[2]);
            finite = finite && fin;
            double dn[3];
            renorm_factors(N, fin ? renorm : 0, p.mag, dn);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                S.ds[k] = dn[k];
                dlast[k] = dn[k];
                if (q == 0) sc->norms[k] = N[k];
            }
        }
        __syncthreads();
    }
    if (valid) A[(size_t)j * nx + i] = S.st[j][lane];
    if (q == 0 && threadIdx.x == 0 && nsteps > 0) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            sc->scale[k] = dlast[k];
            sc->scale_f[k] = (float)dlast[k];
            sc->scale_l[k] = (float)(dlast[k] - (double)sc->scale_f[k]);
        }
        sc->scale_src = 0;
        if (!finite) sc->err |= 1;
        sc->step_idx = step0 + nsteps;
    }
}

}  // namespace sgpe
