// sgpe_batch.cu -- batched form: many independent grids (1D and 2D, uneven
// sizes, uneven physical parameters) advanced together by the same split step
// (arXiv:2009.13507, Sec. 3 and Appendix A) in grouped launches replayed from
// CUDA graphs. Every launch covers all instances through device work lists:
//   x part      either the fused row kernel (pointwise substeps + CN along x,
//               one block per row, one launch per chunk length C) or a
//               pointwise kernel (one block per 128-point tile of any
//               instance) and CN along x (one warp per line, one launch per C;
//               the register kernels are compiled per C)
//   CN along y  one warp per column or column pair (2D instances), one launch per C
//   finalize    one block per instance (norms, renormalisation scale)
// The x part and the warps per block of the sweeps are chosen by
// sgpe_batch_autotune (or set by sgpe_batch_set_tiles).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "../../include/sgpe.h"
#include "sgpe_cn.cuh"
#include "sgpe_kernels.cuh"
#include "sgpe_launch.h"

namespace sgpe {

// Device descriptor of one instance.
struct BInst {
    KParams p;
    long long off;  // element offset of the instance state in the batch state (and mid) buffers
    long long tab;  // element offset of the instance CN tables in the table pool
    int lenx, leny; // table lengths per axis
    int slot0;      // first partial-norm slot of the instance's final sweep
    int nslot;
    int tile0;      // first pointwise / observable tile
    int ntile;
};

// Tables of an instance: [mode 0 imag, 1 real][axis x, y][fa, fg, fp, fq].
template <typename R>
__device__ __forceinline__ Tabs<R> inst_tabs(const typename V2<R>::T* pool, const BInst& I, int mode, int axis) {
    const typename V2<R>::T* b = pool + I.tab + (long long)mode * 4 * (I.lenx + I.leny);
    const int len = axis == 0 ? I.lenx : I.leny;
    if (axis == 1) b += 4 * I.lenx;
    return Tabs<R>{b, b + len, b + 2 * len, b + 3 * len};
}

// Tile t of an instance: 2D tiles are 32 x 4 points, 1D tiles 128 points.
__device__ __forceinline__ void tile_point(const KParams& p, int t, int* ix, int* iy) {
    if (p.dim == 2) {
        const int ntx = (p.nx + 31) / 32;
        *ix = (t % ntx) * 32 + (threadIdx.x & 31);
        *iy = (t / ntx) * 4 + (threadIdx.x >> 5);
    } else {
        *ix = t * 128 + threadIdx.x;
        *iy = 0;
    }
}

template <typename R, bool IMAG>
__global__ void __launch_bounds__(128) kb_pointwise(const typename V2<R>::T* __restrict__ A,
                                                    typename V2<R>::T* __restrict__ B, const BInst* __restrict__ insts,
                                                    const int2* __restrict__ tiles, const DevScalars* __restrict__ scs) {
    const int2 tl = tiles[blockIdx.x];
    const BInst& I = insts[tl.x];
    int ix, iy;
    tile_point(I.p, tl.y, &ix, &iy);
    if (ix >= I.p.nx || iy >= I.p.ny) return;
    pointwise_at<R, IMAG>(A + I.off, B + I.off, I.p, scs + tl.x, kc<R>(I.p, KC_OMEGA), ix, iy, 7);
}

// Fused row kernel (the batched form of k_pwx): one block per row of one
// instance, work entry (instance, row iy, first partial slot or -1). The
// pointwise substeps (pending scale of the instance, SO, CALCNU, HERM) of the
// row's points are staged in shared memory in the lanes' chunk layout, then
// warp j solves the x line of component j. 2D rows go to B for the y sweep; a 1D
// instance is one row, written back to A in place (every read of the row is done
// before the staging barrier) with its three norm partials.
template <typename R, bool IMAG, int C>
__global__ void __launch_bounds__(kPwxThreads, pwx_min_blocks<R, C, IMAG>())
    kb_pwx(typename V2<R>::T* A, typename V2<R>::T* B, const BInst* __restrict__ insts,
           const typename V2<R>::T* __restrict__ pool, const int4* __restrict__ rows,
           const DevScalars* __restrict__ scs, double* partials) {
    using T = typename V2<R>::T;
    extern __shared__ __align__(16) unsigned char kbpwx_smem[];
    T* row = reinterpret_cast<T*>(kbpwx_smem);
    __shared__ R ds[3];
    constexpr int S = 32 * (C + 1);
    constexpr int PPT = (32 * C + kPwxThreads - 1) / kPwxThreads;
    const int4 e = rows[blockIdx.x];
    const BInst& I = insts[e.x];
    const KParams& p = I.p;
    const int iy = e.y, nx = p.nx;
    const int warp = threadIdx.x >> 5;
    PointIn<R> in[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int ix = threadIdx.x + k * kPwxThreads;
        if (ix < nx) pointwise_load<R>(A + I.off, p, ix, iy, p.so_case != 0, in[k]);
    }
    if (threadIdx.x < 3) ds[threadIdx.x] = scale_of<R>(scs + e.x, threadIdx.x);
    __syncthreads();
    const R Ot = kc<R>(p, KC_OMEGA);
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int ix = threadIdx.x + k * kPwxThreads;
        if (ix < nx) {
            cx<R> u[3];
            pointwise_apply<R, IMAG>(in[k], p, ds, Ot, ix, iy, 7, u);
            const int slot = (ix / C) * (C + 1) + (ix % C);
#pragma unroll
            for (int j = 0; j < 3; j++) row[j * S + slot] = pack(u[j]);
        }
    }
    __syncthreads();
    if (warp < 3) {
        const T* r = row + warp * S;
        const Tabs<R> t = inst_tabs<R>(pool, I, IMAG ? 0 : 1, 0);
        T* out = (p.dim == 2 ? B : A) + I.off;
        const size_t base = ((size_t)warp * p.ny + iy) * nx;
        cnx_solve_line<R, IMAG, C>([&](int i) { return unpack(r[(i / C) * (C + 1) + (i % C)]); }, out, base, nx, t,
                                   e.z >= 0 ? partials + e.z + warp : nullptr);
    }
}

// Work entry of the x sweep: (instance, line, partial slot or -1).
template <typename R, bool IMAG, int C>
__global__ void kb_cnx(typename V2<R>::T* A, typename V2<R>::T* B, const BInst* __restrict__ insts,
                       const typename V2<R>::T* __restrict__ pool, const int4* __restrict__ work, int nwork,
                       double* partials) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nwork) return;  // whole warp
    const int4 e = work[w];
    const BInst& I = insts[e.x];
    const Tabs<R> t = inst_tabs<R>(pool, I, IMAG ? 0 : 1, 0);
    typename V2<R>::T* out = (I.p.dim == 2 ? B : A) + I.off;
    cnx_line<R, IMAG, C>(B + I.off, out, I.p, t, e.y, e.z >= 0 ? partials + e.z : nullptr);
}

// Work entry of the y sweep: (instance, component, first column, partial slot).
template <typename R, bool IMAG, int C>
__global__ void kb_cny(typename V2<R>::T* A, const typename V2<R>::T* B, const BInst* __restrict__ insts,
                       const typename V2<R>::T* __restrict__ pool, const int4* __restrict__ work, int nwork,
                       double* partials) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= nwork) return;
    const int4 e = work[w];
    const BInst& I = insts[e.x];
    const Tabs<R> t = inst_tabs<R>(pool, I, IMAG ? 0 : 1, 1);
    cny_cols<R, IMAG, C>(B + I.off, A + I.off, I.p, t, e.y, e.z, partials + e.w);
}

// Shortest axis of a batch instance on the tiled step.
constexpr int kBatchMidMinN = 128;

// Tiled instances (complex64 2D grids of 128..1024 points an axis with even rows,
// the constant-factor form in both time modes): the kernels of the single-grid
// tiled step through work lists. uni holds the instances' constant-factor forms as
// Tabs, [instance][mode][axis].
// Row entry: (instance, row, -, -); one launch per warps-a-line count (blockDim 96 nwl).
template <bool IMAG>
__global__ void __launch_bounds__(96 * kPwxLongMaxGroupWarps, 2)
    kb_pwx_long(const float2* __restrict__ A, float2* __restrict__ B, const BInst* __restrict__ insts,
                const Tabs<float>* __restrict__ uni, const int4* __restrict__ rows,
                const DevScalars* __restrict__ scs) {
    const int4 e = rows[blockIdx.x];
    const BInst& I = insts[e.x];
    f32x2 ds[3];
    float Ot;
    pair_constants(I.p, scs + e.x, nullptr, 7, ds, Ot);
    const Tabs<float> t = uni[4 * e.x + (IMAG ? 0 : 2)];
    pwx_long_row<IMAG, false>(A + I.off, B + I.off, I.p, ds, Ot, t, 7, e.y);
}

// Tile entry: (instance, component j + 4 column tile, row tile, partial slot); one
// launch per halo depth HC. The tile's norm goes to its FP64 partial slot.
template <bool IMAG, int HC>
__global__ void __launch_bounds__(32 * (kTileReal + 2 * HC), (tile_min_blocks<float, HC>()))
    kb_cny_tile(float2* __restrict__ A, const float2* __restrict__ B, const BInst* __restrict__ insts,
                const Tabs<float>* __restrict__ uni, const int4* __restrict__ work, double* partials) {
    const int4 e = work[blockIdx.x];
    const BInst& I = insts[e.x];
    const Tabs<float> t = uni[4 * e.x + (IMAG ? 0 : 2) + 1];
    const df sum = cny_tile<float, IMAG, HC, kTileReal>(B + I.off, A + I.off, I.p, t, e.y & 3, e.y >> 2, e.z, true);
    if (threadIdx.x == 0) partials[e.w] = (double)sum.hi + (double)sum.lo;
}

// One block per instance: sum its partial slots in order, publish norms and the
// next pending scale (imaginary time with renorm != 0), advance its step count.
__global__ void __launch_bounds__(128) kb_finalize(const BInst* __restrict__ insts, const double* partials,
                                                   DevScalars* scs, int imag) {
    __shared__ double red[4 * 3];
    const BInst& I = insts[blockIdx.x];
    double s[3] = {0.0, 0.0, 0.0};
    // slots of component j: [slot0 + j*m, slot0 + (j+1)*m)
    const int m = I.nslot / 3;
    for (int b = threadIdx.x; b < m; b += blockDim.x) {
        const double* q = partials + I.slot0 + b;
        s[0] += __ldcg(q);
        s[1] += __ldcg(q + m);
        s[2] += __ldcg(q + 2 * m);
    }
    block_reduce<3>(s, red);
    if (threadIdx.x == 0) {
        DevScalars* sc = scs + blockIdx.x;
        double N[3] = {s[0] * I.p.cell, s[1] * I.p.cell, s[2] * I.p.cell};
        bool finite = isfinite(N[0]) && isfinite(N[1]) && isfinite(N[2]);
        double d[3];
        renorm_factors(N, (finite && imag) ? I.p.renorm : 0, I.p.mag, d);
        for (int j = 0; j < 3; j++) {
            sc->norms[j] = N[j];
            sc->scale[j] = d[j];
            sc->scale_f[j] = (float)d[j];
            sc->scale_l[j] = (float)(d[j] - (double)sc->scale_f[j]);
        }
        if (!finite) sc->err |= 1;
        sc->step_idx += 1;
    }
}

template <typename R>
__global__ void __launch_bounds__(128) kb_flush(typename V2<R>::T* A, const BInst* __restrict__ insts,
                                                const int2* __restrict__ tiles, const DevScalars* __restrict__ scs) {
    const int2 tl = tiles[blockIdx.x];
    const BInst& I = insts[tl.x];
    int ix, iy;
    tile_point(I.p, tl.y, &ix, &iy);
    if (ix >= I.p.nx || iy >= I.p.ny) return;
    const size_t plane = (size_t)I.p.nx * I.p.ny, c = (size_t)iy * I.p.nx + ix;
    for (int j = 0; j < 3; j++) {
        typename V2<R>::T* a = A + I.off + j * plane + c;
        cx<R> v = ldc<R>(A + I.off, j * plane + c);
        st<R>(a, 0, scl((R)scs[tl.x].scale[j], v));
    }
}

__global__ void kb_reset(DevScalars* scs, int n, int clear_err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        for (int j = 0; j < 4; j++) {
            scs[i].scale[j] = 1.0;
            scs[i].scale_f[j] = 1.0f;
            scs[i].scale_l[j] = 0.0f;
        }
    if (i < n && clear_err) scs[i].err = 0;
}

template <typename R>
__global__ void __launch_bounds__(128) kb_obs_tiles(const typename V2<R>::T* __restrict__ A,
                                                    const BInst* __restrict__ insts, const int2* __restrict__ tiles,
                                                    double* partials) {
    __shared__ double red[4 * NACC];
    const int2 tl = tiles[blockIdx.x];
    const BInst& I = insts[tl.x];
    int ix, iy;
    tile_point(I.p, tl.y, &ix, &iy);
    double v[NACC];
    for (int q = 0; q < NACC; q++) v[q] = 0.0;
    if (ix < I.p.nx && iy < I.p.ny) obs_point<R>(A + I.off, I.p, I.p.omega_t, ix, iy, v);
    block_reduce<NACC>(v, red);
    if (threadIdx.x == 0)
        for (int q = 0; q < NACC; q++) partials[(size_t)blockIdx.x * NACC + q] = v[q];
}

__global__ void __launch_bounds__(128) kb_obs_final(const BInst* __restrict__ insts, const double* partials,
                                                    DevScalars* scs) {
    __shared__ double red[4 * NACC];
    const BInst& I = insts[blockIdx.x];
    double s[NACC];
    for (int q = 0; q < NACC; q++) s[q] = 0.0;
    for (int b = threadIdx.x; b < I.ntile; b += blockDim.x)
        for (int q = 0; q < NACC; q++) s[q] += __ldcg(partials + (size_t)(I.tile0 + b) * NACC + q);
    block_reduce<NACC>(s, red);
    if (threadIdx.x == 0) obs_finish(s, I.p.cell, scs[blockIdx.x].obs, &scs[blockIdx.x].err);
}

}  // namespace sgpe

using namespace sgpe;

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct BGraphKey {
    int imag, count;
    bool operator<(const BGraphKey& o) const { return imag != o.imag ? imag < o.imag : count < o.count; }
};

struct sgpe_batch {
    int n;
    sgpe_precision prec;
    int esz;
    cudaStream_t stream;
    std::vector<sgpe_instance> inst;
    std::vector<BInst> hinst;
    std::vector<int2> tiles;    // every instance's tiles (flush, observables)
    std::vector<int2> pwtiles;  // the tiles of the pointwise kernel (instances on the register path)
    std::map<int, std::vector<int4>> cnx, cny, rows;  // work lists by chunk length (rows: the fused x part)
    // tiled instances (complex64): row entries by warps a line, tile entries by halo depth
    std::vector<char> tiled;
    std::map<int, std::vector<int4>> rows_t, ytile;
    size_t state_elems;
    long long tab_elems;
    int nslots;
    // workspace layout (byte offsets)
    size_t o_inst, o_sc, o_tiles, o_part, o_tab, o_mid, total;
    size_t o_pwtiles, o_uni, o_us;
    std::map<int, size_t> o_cnx, o_cny, o_rows, o_rows_t, o_ytile;
    // bound buffers
    void* psi;
    unsigned char* work;
    // launch shape: x part (0: the fused row kernel; 1, 2 or 4: warps per block of
    // the separate x sweep after the pointwise kernel), warps per block of the y sweep
    int wx, wy;
    std::map<BGraphKey, cudaGraphExec_t> graphs;
    bool graphs_ok;
    char err[512];
};

static sgpe_status bfail(sgpe_batch* b, sgpe_status st, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define BCK(expr, where)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) return bfail(b, SGPE_ECUDA, "%s: %s", where, cudaGetErrorString(e_)); \
    } while (0)

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static void binvalidate(sgpe_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

template <typename R, bool IMAG, int C>
static void kb_pwx_c(dim3 grid, dim3 block, cudaStream_t s, typename V2<R>::T* A, typename V2<R>::T* B,
                     const BInst* I, const typename V2<R>::T* pool, const int4* w, const DevScalars* sc,
                     double* part) {
    kb_pwx<R, IMAG, C><<<grid, block, pwx_smem_bytes<R, C>(), s>>>(A, B, I, pool, w, sc, part);
}

// Shared-memory allowance of the fused row kernels (rows of 1024 points stage 51 KB).
template <typename R, bool IMAG> static cudaError_t kb_pwx_allow() {
    cudaError_t e = cudaSuccess;
    if (!e) e = cudaFuncSetAttribute(kb_pwx<R, IMAG, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pwx_smem_bytes<R, 16>());
    if (!e) e = cudaFuncSetAttribute(kb_pwx<R, IMAG, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pwx_smem_bytes<R, 32>());
    return e;
}

// Enqueue one step for all instances.
template <typename R, bool IMAG>
static cudaError_t benqueue_step(sgpe_batch* b) {
    using T = typename V2<R>::T;
    T* A = (T*)b->psi;
    T* B = (T*)(b->work + b->o_mid);
    const BInst* I = (const BInst*)(b->work + b->o_inst);
    DevScalars* sc = (DevScalars*)(b->work + b->o_sc);
    const int2* tiles = (const int2*)(b->work + b->o_tiles);
    double* part = (double*)(b->work + b->o_part);
    const T* pool = (const T*)(b->work + b->o_tab);
    if (b->wx == 0) {
        for (auto& kv : b->rows) {
            const int4* w = (const int4*)(b->work + b->o_rows[kv.first]);
            const dim3 grid((unsigned)kv.second.size()), block(kPwxThreads);
            switch (kv.first) {
                case 1: kb_pwx_c<R, IMAG, 1>(grid, block, b->stream, A, B, I, pool, w, sc, part); break;
                case 2: kb_pwx_c<R, IMAG, 2>(grid, block, b->stream, A, B, I, pool, w, sc, part); break;
                case 4: kb_pwx_c<R, IMAG, 4>(grid, block, b->stream, A, B, I, pool, w, sc, part); break;
                case 8: kb_pwx_c<R, IMAG, 8>(grid, block, b->stream, A, B, I, pool, w, sc, part); break;
                case 16: kb_pwx_c<R, IMAG, 16>(grid, block, b->stream, A, B, I, pool, w, sc, part); break;
                default: kb_pwx_c<R, IMAG, 32>(grid, block, b->stream, A, B, I, pool, w, sc, part); break;
            }
        }
    } else if (!b->pwtiles.empty()) {
        const int2* pwt = (const int2*)(b->work + b->o_pwtiles);
        kb_pointwise<R, IMAG><<<(unsigned)b->pwtiles.size(), 128, 0, b->stream>>>(A, B, I, pwt, sc);
    }
    if constexpr (std::is_same<R, float>::value) {
        const Tabs<float>* uni = (const Tabs<float>*)(b->work + b->o_uni);
        for (auto& kv : b->rows_t) {
            const int4* w = (const int4*)(b->work + b->o_rows_t[kv.first]);
            const size_t sm = (size_t)3 * 32 * kv.first * kLongS * sizeof(cx<float>);
            kb_pwx_long<IMAG><<<(unsigned)kv.second.size(), 96 * kv.first, sm, b->stream>>>(
                (const float2*)A, (float2*)B, I, uni, w, sc);
        }
    }
    for (auto& kv : b->cnx) {
        if (b->wx == 0) break;  // fused into kb_pwx
        const int4* w = (const int4*)(b->work + b->o_cnx[kv.first]);
        int nw = (int)kv.second.size();
        dim3 grid((nw + b->wx - 1) / b->wx), block(32 * b->wx);
        switch (kv.first) {
            case 1: kb_cnx<R, IMAG, 1><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 2: kb_cnx<R, IMAG, 2><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 4: kb_cnx<R, IMAG, 4><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 8: kb_cnx<R, IMAG, 8><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 16: kb_cnx<R, IMAG, 16><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            default: kb_cnx<R, IMAG, 32><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
        }
    }
    for (auto& kv : b->cny) {
        const int4* w = (const int4*)(b->work + b->o_cny[kv.first]);
        int nw = (int)kv.second.size();
        dim3 grid((nw + b->wy - 1) / b->wy), block(32 * b->wy);
        switch (kv.first) {
            case 1: kb_cny<R, IMAG, 1><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 2: kb_cny<R, IMAG, 2><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 4: kb_cny<R, IMAG, 4><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 8: kb_cny<R, IMAG, 8><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            case 16: kb_cny<R, IMAG, 16><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
            default: kb_cny<R, IMAG, 32><<<grid, block, 0, b->stream>>>(A, B, I, pool, w, nw, part); break;
        }
    }
    if constexpr (std::is_same<R, float>::value) {
        const Tabs<float>* uni = (const Tabs<float>*)(b->work + b->o_uni);
        for (auto& kv : b->ytile) {
            const int4* w = (const int4*)(b->work + b->o_ytile[kv.first]);
            const int hc = kv.first;
            const size_t sm = (size_t)(kTileReal + 2 * hc) * kLongC * 32 * sizeof(cx<float>);
            const dim3 grid((unsigned)kv.second.size()), block(32 * (kTileReal + 2 * hc));
            if (hc == 1)
                kb_cny_tile<IMAG, 1><<<grid, block, sm, b->stream>>>((float2*)A, (const float2*)B, I, uni, w, part);
            else
                kb_cny_tile<IMAG, 2><<<grid, block, sm, b->stream>>>((float2*)A, (const float2*)B, I, uni, w, part);
        }
    }
    kb_finalize<<<b->n, 128, 0, b->stream>>>(I, part, sc, IMAG ? 1 : 0);
    return cudaGetLastError();
}

static cudaError_t benqueue_steps(sgpe_batch* b, int n, bool imag) {
    for (int i = 0; i < n; i++) {
        cudaError_t e;
        if (b->prec == SGPE_C128)
            e = imag ? benqueue_step<double, true>(b) : benqueue_step<double, false>(b);
        else
            e = imag ? benqueue_step<float, true>(b) : benqueue_step<float, false>(b);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static sgpe_status brun(sgpe_batch* b, int nsteps, bool imag) {
    const int G = nsteps < 32 ? nsteps : 32;
    const int reps = G > 0 ? nsteps / G : 0, rem = G > 0 ? nsteps - reps * G : 0;
    cudaGraphExec_t exec = nullptr;
    if (b->graphs_ok && b->stream != nullptr && reps > 0 && G >= 4) {
        BGraphKey key{imag ? 1 : 0, G};
        auto it = b->graphs.find(key);
        if (it != b->graphs.end()) {
            exec = it->second;
        } else {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = benqueue_steps(b, G, imag);
                e = cudaStreamEndCapture(b->stream, &g);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                cudaGetLastError();
                exec = nullptr;
                b->graphs_ok = false;
            } else {
                b->graphs[key] = exec;
            }
        }
    }
    if (exec) {
        for (int r = 0; r < reps; r++) BCK(cudaGraphLaunch(exec, b->stream), "cudaGraphLaunch");
        BCK(benqueue_steps(b, rem, imag), "batch step kernels");
    } else {
        BCK(benqueue_steps(b, nsteps, imag), "batch step kernels");
    }
    return SGPE_OK;
}

template <typename R> static cudaError_t bflush(sgpe_batch* b) {
    using T = typename V2<R>::T;
    const BInst* I = (const BInst*)(b->work + b->o_inst);
    DevScalars* sc = (DevScalars*)(b->work + b->o_sc);
    const int2* tiles = (const int2*)(b->work + b->o_tiles);
    kb_flush<R><<<(unsigned)b->tiles.size(), 128, 0, b->stream>>>((T*)b->psi, I, tiles, sc);
    kb_reset<<<(b->n + 127) / 128, 128, 0, b->stream>>>(sc, b->n, 0);
    return cudaGetLastError();
}

extern "C" {

sgpe_status sgpe_batch_create(sgpe_batch** out, int n, const sgpe_instance* inst, sgpe_precision prec,
                              void* cuda_stream) {
    if (!out) return SGPE_EINVAL;
    *out = nullptr;
    if (n < 1 || !inst) {
        set_thread_error("sgpe_batch_create: need n >= 1 instances");
        return SGPE_EINVAL;
    }
    if (prec == SGPE_CDF) return SGPE_EUNSUPPORTED;
    if (prec != SGPE_C128 && prec != SGPE_C64) return SGPE_EINVAL;
    for (int i = 0; i < n; i++) {
        const sgpe_instance& q = inst[i];
        int ny = q.dim == 1 ? 1 : q.ny;
        double dy = q.dim == 1 ? q.dx : q.dy;
        if ((q.dim != 1 && q.dim != 2) || q.nx < 3 || (q.dim == 2 && ny < 3) || !(q.dx > 0.0) || !(dy > 0.0) ||
            !isfinite(q.dx) || !isfinite(dy)) {
            char m[128];
            snprintf(m, sizeof(m), "sgpe_batch_create: instance %d has an invalid grid", i);
            set_thread_error(m);
            return SGPE_EINVAL;
        }
        if (q.nx > kRegMaxN || ny > kRegMaxN) {
            char m[128];
            snprintf(m, sizeof(m), "sgpe_batch_create: instance %d: lines longer than %d points", i, kRegMaxN);
            set_thread_error(m);
            return SGPE_EUNSUPPORTED;
        }
        if (const char* why = check_params(&q.params)) {
            char m[160];
            snprintf(m, sizeof(m), "sgpe_batch_create: instance %d: %s", i, why);
            set_thread_error(m);
            return SGPE_EINVAL;
        }
        if (q.params.split || q.params.so_mode) {
            char m[160];
            snprintf(m, sizeof(m), "sgpe_batch_create: instance %d: Strang splitting and the SO by Crank-Nicolson "
                     "are single-grid options", i);
            set_thread_error(m);
            return SGPE_EUNSUPPORTED;
        }
    }
    sgpe_batch* b = new (std::nothrow) sgpe_batch();
    if (!b) return SGPE_ENOMEM;
    b->n = n;
    b->prec = prec;
    b->esz = prec == SGPE_C128 ? 16 : 8;
    b->stream = (cudaStream_t)cuda_stream;
    b->inst.assign(inst, inst + n);
    b->psi = nullptr;
    b->work = nullptr;
    b->wx = 0;
    b->wy = 1;
    b->graphs_ok = true;
    b->err[0] = 0;
    long long off = 0, tab = 0;
    int slot = 0;
    for (int i = 0; i < n; i++) {
        sgpe_instance q = inst[i];
        if (q.dim == 1) {
            q.ny = 1;
            q.dy = q.dx;
        }
        BInst I;
        memset(&I, 0, sizeof(I));
        I.p = make_kparams(q.dim, q.nx, q.ny, q.dx, q.dy, &q.params);
        fill_derived(I.p);
        I.off = off;
        off += ((long long)3 * q.nx * q.ny + 63) / 64 * 64;
        I.lenx = table_len(q.nx);
        I.leny = q.dim == 2 ? table_len(q.ny) : 0;
        I.tab = tab;
        tab += 2LL * 4 * (I.lenx + I.leny);
        I.tile0 = (int)b->tiles.size();
        I.ntile = q.dim == 2 ? ceil_div(q.nx, 32) * ceil_div(q.ny, 4) : ceil_div(q.nx, 128);
        // complex64 2D instances of 128..1024 points an axis with even rows take the tiled
        // step when both axes have the constant-factor form in both time modes (from 128
        // points: inside a batch the grouped launches fill the GPU; 64-instance workload
        // 6.87e9 -> 7.49e9 point-steps/s against a 256-point threshold)
        bool tl = prec == SGPE_C64 && q.dim == 2 && q.nx % 2 == 0 && q.nx >= kBatchMidMinN && q.ny >= kBatchMidMinN;
        int hcmax = 0;
        for (int m = 0; m < 2 && tl; m++)
            for (int a = 0; a < 2 && tl; a++) {
                const double h = a == 0 ? q.dx : q.dy, bt = q.params.dt / (4.0 * h * h);
                UniHost u;
                if (Launcher<float>::uni(nullptr, a == 0 ? q.nx : q.ny, m == 0 ? bt : 0.0, m == 0 ? 0.0 : bt, nullptr,
                                         &u) != cudaSuccess ||
                    u.ks <= 0 || (a == 1 && u.hc <= 0))
                    tl = false;
                else if (a == 1)
                    hcmax = std::max(hcmax, u.hc);
            }
        b->tiled.push_back(tl ? 1 : 0);
        for (int t = 0; t < I.ntile; t++) {
            b->tiles.push_back(make_int2(i, t));
            if (!tl) b->pwtiles.push_back(make_int2(i, t));
        }
        const int Cx = chunk_len(q.nx);
        I.slot0 = slot;
        if (tl) {
            const int nwl = long_warps(q.nx);
            for (int r = 0; r < q.ny; r++) b->rows_t[nwl].push_back(make_int4(i, r, 0, 0));
            const int nct = ceil_div(q.nx, 32), nrt = ceil_div(q.ny, kTileRows);
            for (int j = 0; j < 3; j++)
                for (int ct = 0; ct < nct; ct++)
                    for (int rt = 0; rt < nrt; rt++)
                        b->ytile[hcmax].push_back(make_int4(i, j + 4 * ct, rt, slot + (j * nct + ct) * nrt + rt));
            I.nslot = 3 * nct * nrt;
            slot += I.nslot;
        } else if (q.dim == 1) {
            I.nslot = 3;
            for (int l = 0; l < 3; l++) b->cnx[Cx].push_back(make_int4(i, l, slot + l, 0));
            b->rows[Cx].push_back(make_int4(i, 0, slot, 0));
            slot += 3;
        } else {
            for (int l = 0; l < 3 * q.ny; l++) b->cnx[Cx].push_back(make_int4(i, l, -1, 0));
            for (int r = 0; r < q.ny; r++) b->rows[Cx].push_back(make_int4(i, r, -1, 0));
            const int Cy = chunk_len(q.ny);
            const int K = cny_cols_per_warp(Cy, b->esz);
            int cnt = 0;
            for (int j = 0; j < 3; j++)
                for (int col = 0; col < q.nx; col += K) b->cny[Cy].push_back(make_int4(i, j, col, slot + cnt++));
            I.nslot = cnt;
            slot += cnt;
        }
        b->hinst.push_back(I);
    }
    b->state_elems = (size_t)off;
    b->tab_elems = tab;
    b->nslots = slot;
    size_t o = 0;
    b->o_inst = o;
    o = al256(o + sizeof(BInst) * n);
    b->o_sc = o;
    o = al256(o + sizeof(DevScalars) * n);
    b->o_tiles = o;
    o = al256(o + sizeof(int2) * b->tiles.size());
    b->o_pwtiles = o;
    o = al256(o + sizeof(int2) * b->pwtiles.size());
    for (auto& kv : b->rows_t) {
        b->o_rows_t[kv.first] = o;
        o = al256(o + sizeof(int4) * kv.second.size());
    }
    for (auto& kv : b->ytile) {
        b->o_ytile[kv.first] = o;
        o = al256(o + sizeof(int4) * kv.second.size());
    }
    // the constant-factor forms of tiled instances: [instance][mode][axis] Tabs and start corrections
    b->o_uni = o;
    o = al256(o + (prec == SGPE_C64 ? sizeof(Tabs<float>) * 4 * (size_t)n : 0));
    b->o_us = o;
    o = al256(o + (prec == SGPE_C64 ? sizeof(float2) * kUniMaxS * 4 * (size_t)n : 0));
    for (auto& kv : b->cnx) {
        b->o_cnx[kv.first] = o;
        o = al256(o + sizeof(int4) * kv.second.size());
    }
    for (auto& kv : b->cny) {
        b->o_cny[kv.first] = o;
        o = al256(o + sizeof(int4) * kv.second.size());
    }
    for (auto& kv : b->rows) {
        b->o_rows[kv.first] = o;
        o = al256(o + sizeof(int4) * kv.second.size());
    }
    b->o_part = o;
    size_t np = std::max((size_t)3 * b->nslots, (size_t)NACC * b->tiles.size());
    o = al256(o + sizeof(double) * np);
    b->o_tab = o;
    o = al256(o + (size_t)b->esz * b->tab_elems);
    b->o_mid = o;
    o = al256(o + (size_t)b->esz * b->state_elems);
    b->total = o;
    *out = b;
    return SGPE_OK;
}

sgpe_status sgpe_batch_sizes(const sgpe_batch* b, size_t* state_elems, size_t* workspace_bytes) {
    if (!b) return SGPE_EINVAL;
    if (state_elems) *state_elems = b->state_elems;
    if (workspace_bytes) *workspace_bytes = b->total;
    return SGPE_OK;
}

sgpe_status sgpe_batch_offsets(const sgpe_batch* b, size_t* offsets) {
    if (!b || !offsets) return SGPE_EINVAL;
    for (int i = 0; i < b->n; i++) offsets[i] = (size_t)b->hinst[i].off;
    return SGPE_OK;
}

sgpe_status sgpe_batch_bind(sgpe_batch* b, void* psi_dev, void* workspace_dev) {
    if (!b) return SGPE_EINVAL;
    if (!psi_dev || !workspace_dev) return bfail(b, SGPE_EINVAL, "sgpe_batch_bind: null buffer");
    if (((uintptr_t)psi_dev & 15) || ((uintptr_t)workspace_dev & 255))
        return bfail(b, SGPE_EINVAL, "sgpe_batch_bind: psi must be 16-byte and workspace 256-byte aligned");
    binvalidate(b);
    b->psi = psi_dev;
    b->work = (unsigned char*)workspace_dev;
    cudaStream_t s = b->stream;
    BCK(cudaMemcpyAsync(b->work + b->o_inst, b->hinst.data(), sizeof(BInst) * b->n, cudaMemcpyHostToDevice, s), "copy");
    BCK(cudaMemsetAsync(b->work + b->o_sc, 0, sizeof(DevScalars) * b->n, s), "memset");
    BCK(cudaMemcpyAsync(b->work + b->o_tiles, b->tiles.data(), sizeof(int2) * b->tiles.size(), cudaMemcpyHostToDevice,
                        s), "copy");
    for (auto& kv : b->cnx)
        BCK(cudaMemcpyAsync(b->work + b->o_cnx[kv.first], kv.second.data(), sizeof(int4) * kv.second.size(),
                            cudaMemcpyHostToDevice, s), "copy");
    for (auto& kv : b->cny)
        BCK(cudaMemcpyAsync(b->work + b->o_cny[kv.first], kv.second.data(), sizeof(int4) * kv.second.size(),
                            cudaMemcpyHostToDevice, s), "copy");
    for (auto& kv : b->rows)
        BCK(cudaMemcpyAsync(b->work + b->o_rows[kv.first], kv.second.data(), sizeof(int4) * kv.second.size(),
                            cudaMemcpyHostToDevice, s), "copy");
    if (!b->pwtiles.empty())
        BCK(cudaMemcpyAsync(b->work + b->o_pwtiles, b->pwtiles.data(), sizeof(int2) * b->pwtiles.size(),
                            cudaMemcpyHostToDevice, s), "copy");
    for (auto& kv : b->rows_t)
        BCK(cudaMemcpyAsync(b->work + b->o_rows_t[kv.first], kv.second.data(), sizeof(int4) * kv.second.size(),
                            cudaMemcpyHostToDevice, s), "copy");
    for (auto& kv : b->ytile)
        BCK(cudaMemcpyAsync(b->work + b->o_ytile[kv.first], kv.second.data(), sizeof(int4) * kv.second.size(),
                            cudaMemcpyHostToDevice, s), "copy");
    if (b->prec == SGPE_C64) {
        // tiled instances: the constant-factor forms (start corrections into the workspace)
        std::vector<Tabs<float>> ut(4 * (size_t)b->n);
        memset(ut.data(), 0, sizeof(Tabs<float>) * ut.size());
        for (int i = 0; i < b->n; i++) {
            if (!b->tiled[i]) continue;
            const BInst& I = b->hinst[i];
            for (int m = 0; m < 2; m++)
                for (int a = 0; a < 2; a++) {
                    const size_t k = 4 * (size_t)i + 2 * m + a;
                    const double h = a == 0 ? I.p.dx : I.p.dy, bt = I.p.dt / (4.0 * h * h);
                    void* sdev = b->work + b->o_us + sizeof(float2) * kUniMaxS * k;
                    UniHost u;
                    BCK(Launcher<float>::uni(s, a == 0 ? I.p.nx : I.p.ny, m == 0 ? bt : 0.0, m == 0 ? 0.0 : bt, sdev,
                                             &u),
                        "constant-factor form");
                    Tabs<float>& t = ut[k];
                    t.ug = {(float)u.gr, (float)u.gi};
                    t.ug16 = {(float)u.g16r, (float)u.g16i};
                    t.uc = {(float)u.cr, (float)u.ci};
                    t.uk = {(float)u.kr, (float)u.ki};
                    for (int q = 0; q < 16; q++) t.upow[q] = {(float)u.pr[q], (float)u.pi[q]};
                    t.us = (const float2*)u.s;
                    t.uks = u.ks;
                    t.unlev = u.nlev;
                }
        }
        BCK(cudaMemcpyAsync(b->work + b->o_uni, ut.data(), sizeof(Tabs<float>) * ut.size(), cudaMemcpyHostToDevice,
                            s),
            "copy");
        BCK(cudaStreamSynchronize(s), "sync");  // the host tables must outlive the copy
        for (int imag = 0; imag < 2; imag++) {
            const size_t sm1 = (size_t)(kTileReal + 2) * kLongC * 32 * sizeof(cx<float>);
            const size_t sm2 = (size_t)(kTileReal + 4) * kLongC * 32 * sizeof(cx<float>);
            BCK(cudaFuncSetAttribute(imag ? kb_cny_tile<true, 1> : kb_cny_tile<false, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1),
                "kernel attributes");
            BCK(cudaFuncSetAttribute(imag ? kb_cny_tile<true, 2> : kb_cny_tile<false, 2>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2),
                "kernel attributes");
        }
    }
    if (b->prec == SGPE_C128) {
        BCK((kb_pwx_allow<double, true>()), "kernel attributes");
        BCK((kb_pwx_allow<double, false>()), "kernel attributes");
    } else {
        BCK((kb_pwx_allow<float, true>()), "kernel attributes");
        BCK((kb_pwx_allow<float, false>()), "kernel attributes");
    }
    DevScalars* sc = (DevScalars*)(b->work + b->o_sc);
    kb_reset<<<(b->n + 127) / 128, 128, 0, s>>>(sc, b->n, 1);
    BCK(cudaGetLastError(), "reset");
    // COEF for every instance, both time modes and axes
    for (int i = 0; i < b->n; i++) {
        const BInst& I = b->hinst[i];
        for (int m = 0; m < 2; m++)
            for (int a = 0; a < I.p.dim; a++) {
                const int len = a == 0 ? I.lenx : I.leny;
                const int nn = a == 0 ? I.p.nx : I.p.ny;
                const double h = a == 0 ? I.p.dx : I.p.dy;
                long long base = I.tab + (long long)m * 4 * (I.lenx + I.leny) + (a == 1 ? 4LL * I.lenx : 0);
                unsigned char* t = b->work + b->o_tab + (size_t)b->esz * base;
                double bt = I.p.dt / (4.0 * h * h);
                double bre = m == 0 ? bt : 0.0, bim = m == 0 ? 0.0 : bt;
                size_t L = (size_t)b->esz * len;
                cudaError_t e = b->prec == SGPE_C128
                                    ? Launcher<double>::coef(s, t, t + L, t + 2 * L, t + 3 * L, nn, bre, bim)
                                    : Launcher<float>::coef(s, t, t + L, t + 2 * L, t + 3 * L, nn, bre, bim);
                BCK(e, "COEF kernel");
            }
    }
    BCK(cudaStreamSynchronize(s), "sync");  // host work lists must outlive the copies
    return SGPE_OK;
}

sgpe_status sgpe_batch_load_state(sgpe_batch* b, const void* psi_dev) {
    if (!b || !psi_dev) return SGPE_EINVAL;
    if (!b->psi) return bfail(b, SGPE_ESTATE, "no buffers bound");
    BCK(cudaMemcpyAsync(b->psi, psi_dev, (size_t)b->esz * b->state_elems, cudaMemcpyDeviceToDevice, b->stream),
        "load_state");
    kb_reset<<<(b->n + 127) / 128, 128, 0, b->stream>>>((DevScalars*)(b->work + b->o_sc), b->n, 1);
    BCK(cudaGetLastError(), "reset");
    return SGPE_OK;
}

sgpe_status sgpe_batch_step_imag(sgpe_batch* b, int nsteps) {
    if (!b) return SGPE_EINVAL;
    if (!b->psi) return bfail(b, SGPE_ESTATE, "no buffers bound");
    if (nsteps < 0) return bfail(b, SGPE_EINVAL, "nsteps < 0");
    return nsteps ? brun(b, nsteps, true) : SGPE_OK;
}

sgpe_status sgpe_batch_step_real(sgpe_batch* b, int nsteps) {
    if (!b) return SGPE_EINVAL;
    if (!b->psi) return bfail(b, SGPE_ESTATE, "no buffers bound");
    if (nsteps < 0) return bfail(b, SGPE_EINVAL, "nsteps < 0");
    return nsteps ? brun(b, nsteps, false) : SGPE_OK;
}

sgpe_status sgpe_batch_energy(sgpe_batch* b, double* out) {
    if (!b || !out) return SGPE_EINVAL;
    if (!b->psi) return bfail(b, SGPE_ESTATE, "no buffers bound");
    BCK(b->prec == SGPE_C128 ? bflush<double>(b) : bflush<float>(b), "flush");
    const BInst* I = (const BInst*)(b->work + b->o_inst);
    const int2* tiles = (const int2*)(b->work + b->o_tiles);
    double* part = (double*)(b->work + b->o_part);
    DevScalars* sc = (DevScalars*)(b->work + b->o_sc);
    if (b->prec == SGPE_C128)
        kb_obs_tiles<double><<<(unsigned)b->tiles.size(), 128, 0, b->stream>>>((const double2*)b->psi, I, tiles, part);
    else
        kb_obs_tiles<float><<<(unsigned)b->tiles.size(), 128, 0, b->stream>>>((const float2*)b->psi, I, tiles, part);
    kb_obs_final<<<b->n, 128, 0, b->stream>>>(I, part, sc);
    BCK(cudaGetLastError(), "observables");
    std::vector<DevScalars> h(b->n);
    BCK(cudaMemcpyAsync(h.data(), sc, sizeof(DevScalars) * b->n, cudaMemcpyDeviceToHost, b->stream), "copy");
    BCK(cudaStreamSynchronize(b->stream), "sync");
    int bad = -1;
    for (int i = 0; i < b->n; i++) {
        memcpy(out + (size_t)SGPE_NOBS * i, h[i].obs, SGPE_NOBS * sizeof(double));
        if (h[i].err && bad < 0) bad = i;
    }
    if (bad >= 0) {
        for (int i = 0; i < b->n; i++) BCK(cudaMemsetAsync(&sc[i].err, 0, sizeof(int), b->stream), "clear err");
        return bfail(b, SGPE_ENONFINITE, "instance %d: non-finite norm", bad);
    }
    return SGPE_OK;
}

sgpe_status sgpe_batch_autotune(sgpe_batch* b, int nsteps, int* choice) {
    if (!b) return SGPE_EINVAL;
    if (!b->psi) return bfail(b, SGPE_ESTATE, "no buffers bound");
    if (nsteps < 1) return bfail(b, SGPE_EINVAL, "nsteps < 1");
    const int candx[4] = {0, 1, 2, 4}, cand[3] = {1, 2, 4};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int bx = 0, by = 1;
    for (int ix = 0; ix < 4; ix++)
        for (int iy = 0; iy < 3; iy++) {
            b->wx = candx[ix];
            b->wy = cand[iy];
            binvalidate(b);
            BCK(benqueue_steps(b, 1, true), "warm-up");
            BCK(cudaEventRecord(e0, b->stream), "event");
            BCK(benqueue_steps(b, nsteps, true), "tune steps");
            BCK(cudaEventRecord(e1, b->stream), "event");
            BCK(cudaEventSynchronize(e1), "sync");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bx = candx[ix];
                by = cand[iy];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->wx = bx;
    b->wy = by;
    binvalidate(b);
    kb_reset<<<(b->n + 127) / 128, 128, 0, b->stream>>>((DevScalars*)(b->work + b->o_sc), b->n, 1);
    BCK(cudaStreamSynchronize(b->stream), "sync");
    if (choice) {
        choice[0] = bx;
        choice[1] = by;
    }
    return SGPE_OK;
}

sgpe_status sgpe_batch_set_tiles(sgpe_batch* b, int x, int y) {
    if (!b) return SGPE_EINVAL;
    if ((x != 0 && x != 1 && x != 2 && x != 4) || (y != 1 && y != 2 && y != 4))
        return bfail(b, SGPE_EINVAL, "sgpe_batch_set_tiles: x in {0, 1, 2, 4}, y in {1, 2, 4}");
    b->wx = x;
    b->wy = y;
    binvalidate(b);
    return SGPE_OK;
}

int sgpe_batch_launches_per_step(const sgpe_batch* b) {
    if (!b) return 0;
    const int t = (int)b->rows_t.size() + (int)b->ytile.size();
    if (b->wx == 0) return 1 + (int)b->rows.size() + (int)b->cny.size() + t;
    return 1 + (b->pwtiles.empty() ? 0 : 1) + (int)b->cnx.size() + (int)b->cny.size() + t;
}

const char* sgpe_batch_last_error(const sgpe_batch* b) { return b ? b->err : "null batch"; }

sgpe_status sgpe_batch_destroy(sgpe_batch* b) {
    if (!b) return SGPE_OK;
    binvalidate(b);
    delete b;
    return SGPE_OK;
}

}  // extern "C"
