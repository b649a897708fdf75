// sgpe_launch.h -- host-side launch interface between the C-ABI layer and the
// per-precision kernel translation units (internal; not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <utility>

#include "../../include/sgpe.h"
#include "sgpe_device.cuh"

namespace sgpe {

struct KParams;
struct DevScalars;
struct SoCnLines;

// Launch a step kernel with programmatic stream serialization: its blocks may
// be scheduled before the previous kernel on the stream completes; the kernel
// itself waits (pdl_wait) before reading what that kernel wrote.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// One launch of a single thread-block cluster of `cluster` CTAs (grid.x == cluster).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cluster(void (*kernel)(KArgs...), unsigned cluster, dim3 block, size_t smem,
                                  cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch geometry shared by the API layer (buffer sizing) and the launchers.
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
// Chunk length (points per lane) of a line of n points: for n <= 1024 the line
// is split over the 32 lanes of one warp, chunk = the next power of two of
// ceil(n/32) (register kernels, compile-time chunk); longer lines are held by a
// group of long_warps(n) warps with kLongC points a lane.
constexpr int kRegMaxN = 1024;
// Longest 1D line of the complex128 cluster step loop (8 CTAs of 32 points).
constexpr int kCl1dMaxN = 256;
inline int chunk_len(int n) {
    if (n > kRegMaxN) return kLongC;
    int c = ceil_div(n, 32);
    int p = 1;
    while (p < c) p <<= 1;
    return p;
}
// Warps of the group that holds a line longer than kRegMaxN points (kLongC points a lane).
inline int long_warps(int n) { return ceil_div(n, 32 * kLongC); }
// Entries of each coefficient table of an n-point axis (padded with zeros past n).
inline int table_len(int n) { return n > kRegMaxN ? 32 * kLongC * long_warps(n) : 32 * chunk_len(n); }
// Columns per warp of the register y sweep (must match CnShape<C>::K).
inline int cny_cols_per_warp(int C, int esz) { return (esz == 8 && C <= 8) ? 2 : 1; }
constexpr int kObsAcc = 11;
constexpr int kNormBlocks = 304;

struct Geometry {
    int dim, nx, ny, esz;
    int wx;  // lines longer than kRegMaxN: warps per block (one line) of the x sweep
    int wy;  // lines longer than kRegMaxN: columns per block (1, 2 or 4) of the y sweep
    bool reg_x, reg_y;  // register-chunk kernels (lines of at most kRegMaxN points)
    bool fused;         // 2D with register x lines: pointwise + CN-x in one kernel
    size_t smem_x, smem_y;
    int blocks_x, blocks_y, blocks_obs, blocks_norm;
    int blocks_yt;  // long columns (and tiled grids): blocks (= norm partials) of the row-tiled y sweep
    int tile_rt;    // chunks of 16 rows that a y tile writes (kTileReal, or kTileRealShort on short columns)
    bool tiled;     // 2D grid of kMidMinN (kMidMinN16)..kRegMaxN points an axis: its steps take the kernels of long
                    // lines (complex64: fused pointwise + x sweep; double-float: pointwise kernel and the
                    // constant-factor x sweep; then the row-tiled y sweep) where the constant-factor form
                    // applies
};
// Shortest axis of a grid that the tiled step serves: complex64 (8-byte elements;
// lines of more than 128 points take 8-point register chunks, slower than the tiles:
// measured at 160, 192 and 224 points, while 128 points stay faster on the register
// kernels) and double-float (16-byte; its register path measured faster on
// 256-point lines).
constexpr int kMidMinN = 129;
constexpr int kMidMinN16 = 320;

Geometry make_geometry(int dim, int nx, int ny, int esz);

// Constant-factor form of a long line's Crank-Nicolson solve (Tabs::uks),
// computed on the host in FP64 when the parameters are set.
struct UniHost {
    double gr, gi, g16r, g16i;  // ug, ug^16
    double cr, ci, kr, ki;      // uc, uk
    double pr[16], pi[16];      // ug^(k+1) (imaginary time: pi = pr)
    int ks;                     // entries of s (0: the line uses the tables)
    int nlev;                   // carry-scan levels
    int hc;                     // halo chunks of the row-tiled y sweep (0: not applicable)
    const void* s;              // device: s_i, i < ks, in the state's element type
};
// The coefficient tables of one axis and time mode, and their constant-factor form.
struct TabSet {
    void* t[4];  // device: fa, fg, fp, fq
    UniHost u;
};

// Whether the y sweep of these tables runs in row tiles (k_cn_y_tile: long
// columns, the constant-factor form with a short carry reach, in != out).
inline bool y_tiled(const Geometry& g, const TabSet& ty, const void* in, const void* out) {
    return g.dim == 2 && (!g.reg_y || g.tiled) && ty.u.ks > 0 && ty.u.hc > 0 && ty.u.ks <= kLongC * g.tile_rt &&
           in != out;
}
// Norm partials that the step's y sweep (in -> out) leaves.
inline int y_parts(const Geometry& g, const TabSet& ty, const void* in, const void* out) {
    return y_tiled(g, ty, in, out) ? g.blocks_yt : g.blocks_y;
}
// Whether the 2D step of a complex64 grid runs its pointwise substeps and x sweep
// in one kernel (k_pwx_long: even rows longer than kRegMaxN and of at most 2048
// points, or the rows of a tiled grid; the constant-factor x solve).
inline bool pwx_long_fits(const Geometry& g, const TabSet& tx) {
    return g.dim == 2 && g.esz == 8 && (!g.reg_x || g.tiled) && g.nx % 2 == 0 && long_warps(g.nx) <= 4 &&
           tx.u.ks > 0;
}
// A step of a tiled grid (Geometry::tiled) on the kernels of long lines: both axes
// in the constant-factor form (which complex128 never takes), the row tiles reaching
// the y carries.
inline bool tiled_step(const Geometry& g, const TabSet& tx, const TabSet& ty) {
    return g.tiled && tx.u.ks > 0 && ty.u.ks > 0 && ty.u.hc > 0 && ty.u.ks <= kLongC * g.tile_rt;
}
// The x sweep of a tiled grid on the constant-factor long-line kernel.
inline bool x_tiled(const Geometry& g, const TabSet& tx) { return g.dim == 2 && g.tiled && tx.u.ks > 0; }
// Longest start correction of the constant-factor form (entries of s).
constexpr int kUniMaxS = 512;

template <typename R> struct Launcher {
    static cudaError_t setup();
    static cudaError_t pointwise(cudaStream_t s, bool imag, const void* A, void* B, const KParams& p,
                                 const DevScalars* sc, const double* omega_tab, int mask);
    // The whole loop of nsteps 1D steps in one block (lines of at most 1024
    // points), the state in shared memory; A is read at the start and written
    // at the end.
    static cudaError_t step1d(cudaStream_t s, bool imag, void* A, const KParams& p, DevScalars* sc,
                              const double* omega_tab, const void* const* tabs_x, int nsteps, int renorm);
    // Fused pointwise substeps + CN along x of a 2D grid (Geometry::fused): A -> B.
    // partials / m / renorm: the previous y sweep's norm partials (m per component)
    // and the renormalisation mode, for the pending scale (DevScalars::scale_src).
    static cudaError_t pwx(cudaStream_t s, bool imag, const void* A, void* B, const KParams& p, const DevScalars* sc,
                           const double* omega_tab, const void* const* tabs_x, const double* partials, int m,
                           int renorm);
    // cn_x / cn_y write per-block FP64 norm partials when last / finalize is set
    // (the step's final sweep); finalize_step then reduces them.
    static cudaError_t cn_x(cudaStream_t s, bool imag, bool last, const void* in, void* out, const KParams& p,
                            const TabSet& tabs, const Geometry& g, double* partials, DevScalars* sc, int renorm,
                            int advance);
    // head_scale (register y sweep of the fused 2D step): the next step's head
    // kernel derives the pending scale from this sweep's partials; the sweep
    // marks that and advances the step counter by advance (no finalize_step).
    static cudaError_t cn_y(cudaStream_t s, bool imag, const void* in, void* out, const KParams& p,
                            const TabSet& tabs, const Geometry& g, double* partials, DevScalars* sc, int renorm,
                            int advance, int finalize, bool head_scale = false);
    // Fused pointwise substeps + CN along x of a 2D complex64 grid (pwx_long_fits):
    // A -> B. partials (nullable) / m / renorm: the previous row-tiled y sweep's norm
    // partials (m per component) for the pending scale (DevScalars::scale_src).
    static cudaError_t pwx_long(cudaStream_t s, bool imag, const void* A, void* B, const KParams& p,
                                const DevScalars* sc, const double* omega_tab, const TabSet& tabs_x, int mask,
                                const double* partials = nullptr, int m = 0, int renorm = 0);
    static cudaError_t coef(cudaStream_t s, void* fa, void* fg, void* fp, void* fq, int n, double bre, double bim);
    // The constant-factor form of an n-point line with bt = bre + i bim: fills u and
    // copies s to s_dev (kUniMaxS entries of room; s_dev null: no copy); u->ks = 0
    // where the correction would be longer than that (and always for complex128).
    static cudaError_t uni(cudaStream_t s, int n, double bre, double bim, void* s_dev, UniHost* u);
    static cudaError_t flush(cudaStream_t s, void* A, size_t plane, const DevScalars* sc);
    // advance: also move the step counter on (the last kernel of a step).
    static cudaError_t norms(cudaStream_t s, const void* A, size_t plane, double cell, int renorm, double mag,
                             double* partials, DevScalars* sc, int advance = 0);
    // SO substep by Crank-Nicolson on one family of lines (lines of at most
    // kRegMaxN points); tabs_p / tabs_m: the skew tables of m = +1 / -1.
    static cudaError_t socn(cudaStream_t s, const void* in, void* out, const SoCnLines& L, const void* const* tabs_p,
                            const void* const* tabs_m, const DevScalars* sc, int scale);
    static cudaError_t coef_skew(cudaStream_t s, void* fa, void* fg, void* fp, void* fq, int n, double are,
                                 double aim);
    static cudaError_t observables(cudaStream_t s, const void* A, const KParams& p, double omega_t,
                                   double* partials, DevScalars* sc);
};

cudaError_t reset_scale(cudaStream_t s, DevScalars* sc);

// Device complex128 [n] -> double-float layout [n] (hi, lo per real part).
cudaError_t cdf_from_c128(cudaStream_t s, const void* src, void* dst, size_t n);

// End of a step: reduce the last sweep's nblk norm partials, publish N_j and the
// next pending scale, advance the step counter (one block).
cudaError_t finalize_step(cudaStream_t s, const double* partials, int nblk, double cell, int renorm, double mag,
                          int advance, DevScalars* sc, int part_df);

// Validation of sgpe_params (nullptr when valid, else the reason) and the kernel
// constants of one grid.
const char* check_params(const sgpe_params* p);
KParams make_kparams(int dim, int nx, int ny, double dx, double dy, const sgpe_params* p);

// Store the message that sgpe_last_error(NULL) returns on this host thread.
void set_thread_error(const char* msg);

// Internal view of a single-grid context for the adjoint translation unit
// (filled by ctx_view in sgpe_api.cu).
struct CtxView {
    int dim, nx, ny, esz;
    bool dbl;
    sgpe_precision prec;
    cudaStream_t stream;
    void* psi;
    void* mid;
    DevScalars* sc;
    const TabSet* tabs_real;  // [axis], bt = i dt/(4h^2)
    const TabSet* tabs_adj;   // [axis], bt = -i dt/(4h^2)
    const Geometry* geo;
    KParams kp;
    double* partials;
    bool ready;
};
bool ctx_view(sgpe_ctx* c, CtxView* v);
sgpe_status ctx_fail(sgpe_ctx* c, sgpe_status st, const char* msg);
cudaError_t ctx_flush(sgpe_ctx* c);

}  // namespace sgpe
