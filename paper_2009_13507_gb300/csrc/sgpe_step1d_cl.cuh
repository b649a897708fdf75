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
// The two halves of a barrier that only says "this CTA runs" (no ordering):
// a CTA may store into a peer's shared memory once it has passed this wait.
__device__ __forceinline__ void cl_arrive_relaxed() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
    __syncwarp();
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
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

// CALCNU factor of component j (the exponent of calcnu_point_dt) applied to u;
// rp, r0, rm: the densities |psi_j|^2 of the three components at the point.
template <bool IMAG>
__device__ __forceinline__ cx<double> calcnu_comp(int j, cx<double> u, double rp, double r0, double rm, double Vn,
                                                  const KParams& p) {
    const double base = fma(p.kd[KC_NC0], rp + r0 + rm, Vn);
    const double nc2 = p.kd[KC_NC2];
    const double x = j == 0 ? fma(nc2, rp - rm + r0, base) : j == 1 ? fma(nc2, rp + rm, base)
                                                                    : fma(nc2, rm - rp + r0, base);
    if (IMAG) return scl(exp_small(x), u);
    double s, c;
    sincos_small(x, &s, &c);
    return mul(cx<double>{c, s}, u);
}

// The off-diagonal entries of the HERM matrix at a point (herm_point):
// a = c2 psi_-^* psi_0 + Ot, b = c2 psi_0^* psi_+ + Ot.
__device__ __forceinline__ cx<double> herm_a(const cx<double> (&u)[3], double c2, double Ot) {
    const cx<double> a = cmul(u[2], u[1]);
    return {fma(c2, a.re, Ot), c2 * a.im};
}
__device__ __forceinline__ cx<double> herm_b(const cx<double> (&u)[3], double c2, double Ot) {
    const cx<double> b = cmul(u[1], u[0]);
    return {fma(c2, b.re, Ot), c2 * b.im};
}

// HERM update of component j (the formulas of herm_point for that component)
// from the point's values u and its matrix entries a, b.
template <bool IMAG>
__device__ __forceinline__ cx<double> herm_comp(int j, const cx<double> (&u)[3], cx<double> a, cx<double> b,
                                                const KParams& p) {
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
    double2 st[3][32];   // the CTA's slice of the three lines (raw state)
    double2 xX[3][32];   // SO: raw differences of each component
    double xr[3][32];    // densities after SO (for CALCNU)
    double2 xb[3][32];   // values after CALCNU (for HERM)
    double2 xab[2][32];  // the HERM entries a (from warp 0) and b (from warp 2)
    // x sweep: the CTAs' segment maps y_end = A y_in + B (forward) and
    // w_start = A w_next + B (backward); the factors A depend on the tables only
    double2 fAs[kCl1dMaxQ], bAs[kCl1dMaxQ];
    double2 fB[3][kCl1dMaxQ], bB[3][kCl1dMaxQ];
    // weights of the earlier (forward) / later (backward) segments' B in this
    // CTA's incoming carry, nearest first, cut where they fall below 2^-64
    double2 wf[kCl1dMaxQ], wb[kCl1dMaxQ];
    int nwf, nwb;
    double part[3][kCl1dMaxQ];  // norm partials of the cluster's CTAs
    double Nc[3];               // the summed norms
    double ds[3];
};

constexpr int kScanLv = 5;  // levels of a full 32-lane scan

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
    cl_arrive_relaxed();  // matched by the cl_wait before the first store into a peer
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
    // The x sweep's scan factors depend on the tables only: the factor each lane
    // applies at each level (fw, bw), the number of levels (see tiny_carry) and
    // the lane's composed factor, once for all steps.
    cx<double> fw[kScanLv], bw[kScanLv], fAc, bAc;
    int nlf = kScanLv, nlb = kScanLv;
    {
        cx<double> a = fg;
#pragma unroll
        for (int l = 0; l < kScanLv; l++) {
            const int off = 1 << l;
            fw[l] = a;
            const cx<double> ap = shup(a, off);
            if (lane >= off) a = tmul<IMAG>(a, ap);
            if (scan_done(lane < 2 * off, a)) {
                nlf = l + 1;
                break;
            }
        }
        fAc = a;
        a = fg;
#pragma unroll
        for (int l = 0; l < kScanLv; l++) {
            const int off = 1 << l;
            bw[l] = a;
            const cx<double> an = shdn(a, off);
            if (lane + off < 32) a = tmul<IMAG>(a, an);
            if (scan_done(lane + 2 * off >= 32, a)) {
                nlb = l + 1;
                break;
            }
        }
        bAc = a;
    }
    const cx<double> fAu = shup(fAc, 1), bAd = shdn(bAc, 1);  // the neighbouring lanes' composed factors
    cl_wait();  // every CTA of the cluster runs
    if (j == 0 && lane == 31)
        for (unsigned r = 0; r < Q; r++) *cl_map(&S.fAs[q], r) = pack(fAc);
    if (j == 0 && lane == 0)
        for (unsigned r = 0; r < Q; r++) *cl_map(&S.bAs[q], r) = pack(bAc);
    __syncthreads();
    cl_sync();  // every CTA has loaded its slice (neighbours may be read) and published its factors
    if (threadIdx.x == 0) {
        // forward carry into CTA q: sum over r of wf[r] B(q - 1 - r), wf[r] = prod_{k<r} A(q - 1 - k)
        cx<double> w = {1.0, 0.0};
        int n = 0;
        for (int r = 0; r < (int)q; r++) {
            if (r > 0) {
                w = tmul<IMAG>(w, unpack(S.fAs[q - r]));
                if (tiny_carry(w.re) && tiny_carry(w.im)) break;
            }
            S.wf[r] = pack(w);
            n = r + 1;
        }
        S.nwf = n;
        // backward carry into CTA q: sum over r of wb[r] B(q + 1 + r), wb[r] = prod_{k<r} A(q + 1 + k)
        w = {1.0, 0.0};
        n = 0;
        for (int r = 0; r + (int)q + 1 < (int)Q; r++) {
            if (r > 0) {
                w = tmul<IMAG>(w, unpack(S.bAs[q + r]));
                if (tiny_carry(w.re) && tiny_carry(w.im)) break;
            }
            S.wb[r] = pack(w);
            n = r + 1;
        }
        S.nwb = n;
    }
    __syncthreads();
    const int nwf = S.nwf, nwb = S.nwb;
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
        S.xr[j][lane] = nrm(u);
        __syncthreads();
        u = calcnu_comp<IMAG>(j, u, S.xr[0][lane], S.xr[1][lane], S.xr[2][lane], Vn, p);
        S.xb[j][lane] = pack(u);
        __syncthreads();
        const cx<double> w[3] = {unpack(S.xb[0][lane]), unpack(S.xb[1][lane]), unpack(S.xb[2][lane])};
        if (j == 0) S.xab[0][lane] = pack(herm_a(w, c2, Ot));
        if (j == 2) S.xab[1][lane] = pack(herm_b(w, c2, Ot));
        __syncthreads();
        u = herm_comp<IMAG>(j, w, unpack(S.xab[0][lane]), unpack(S.xab[1][lane]), p);
        const cx<double> x = valid ? u : zero;  // the CN right-hand side
        // --- CN along x, forward: y_i = fa_i x_i + fg_i y_{i-1}
        const cx<double> yl = tmul<IMAG>(fa, x);
        cx<double> sB = yl;
#pragma unroll
        for (int l = 0; l < kScanLv; l++) {
            if (l >= nlf) break;
            const int off = 1 << l;
            const cx<double> Bp = shup(sB, off);
            if (lane >= off) sB = tfma<IMAG>(fw[l], Bp, sB);
        }
        if (lane == 31)
            for (unsigned r = 0; r < Q; r++) *cl_map(&S.fB[j][q], r) = pack(sB);
        cl_sync();
        // y at the last point of the previous CTAs' segments
        cx<double> cinC = zero;
        if (q > 0) {
            cinC = unpack(S.fB[j][q - 1]);
            for (int r = 1; r < nwf; r++) cinC = tfma<IMAG>(unpack(S.wf[r]), unpack(S.fB[j][q - 1 - r]), cinC);
        }
        const cx<double> Bu = shup(sB, 1);
        const cx<double> yprev = lane == 0 ? cinC : tfma<IMAG>(fAu, cinC, Bu);
        const cx<double> y = tfma<IMAG>(fg, yprev, yl);
        // --- backward: w_i = y_i + fg_i w_{i+1}
        sB = y;
#pragma unroll
        for (int l = 0; l < kScanLv; l++) {
            if (l >= nlb) break;
            const int off = 1 << l;
            const cx<double> Bn = shdn(sB, off);
            if (lane + off < 32) sB = tfma<IMAG>(bw[l], Bn, sB);
        }
        if (lane == 0)
            for (unsigned r = 0; r < Q; r++) *cl_map(&S.bB[j][q], r) = pack(sB);
        cl_sync();
        cx<double> cbC = zero;
        if (q + 1 < Q) {
            cbC = unpack(S.bB[j][q + 1]);
            for (int r = 1; r < nwb; r++) cbC = tfma<IMAG>(unpack(S.wb[r]), unpack(S.bB[j][q + 1 + r]), cbC);
        }
        const cx<double> Bn = shdn(sB, 1);
        const cx<double> wnext = lane == 31 ? cbC : tfma<IMAG>(bAd, cbC, Bn);
        const cx<double> wv = tfma<IMAG>(fg, wnext, y);
        const cx<double> o = valid ? cx<double>{fma(2.0, wv.re, -x.re), fma(2.0, wv.im, -x.im)} : zero;
        S.st[j][lane] = pack(o);
        // --- norm partials to every CTA; every CTA sums them in the same order
        const double pn = warp_sum(nrm(o));
        if (lane == 0)
            for (unsigned r = 0; r < Q; r++) *cl_map(&S.part[j][q], r) = pn;
        cl_sync();
        {
            double v = lane < (int)Q ? S.part[j][lane] : 0.0;  // Q <= 8: lanes 0..7
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            if (lane == 0) S.Nc[j] = v * p.cell;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double N[3] = {S.Nc[0], S.Nc[1], S.Nc[2]};
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
