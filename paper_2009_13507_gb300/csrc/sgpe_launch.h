// sgpe_launch.h -- host-side launch interface between the C-ABI layer and the
// per-precision kernel translation units (internal; not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace sgpe {

struct KParams;
struct DevScalars;

// Launch geometry shared by the API layer (buffer sizing) and the launchers.
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
inline int chunk_len(int n) { return ceil_div(n, 32); }
inline int chunk_stride(int n) { return chunk_len(n) | 1; }
constexpr int kObsAcc = 11;
constexpr int kNormBlocks = 304;

struct Geometry {
    int dim, nx, ny, esz;
    int wx;  // warps (lines) per block of the x sweep
    int wy;  // warps (columns) per block of the y sweep
    size_t smem_x, smem_y;
    int blocks_x, blocks_y, blocks_obs, blocks_norm;
};

Geometry make_geometry(int dim, int nx, int ny, int esz);

template <typename R> struct Launcher {
    static cudaError_t setup();
    static cudaError_t pointwise(cudaStream_t s, bool imag, const void* A, void* B, const KParams& p,
                                 const DevScalars* sc, const double* omega_tab, int mask);
    static cudaError_t cn_x(cudaStream_t s, bool imag, bool last, const void* in, void* out, const KParams& p,
                            const void* const* tabs, const Geometry& g, double* partials, DevScalars* sc, int renorm,
                            int advance);
    static cudaError_t cn_y(cudaStream_t s, bool imag, const void* in, void* out, const KParams& p,
                            const void* const* tabs, const Geometry& g, double* partials, DevScalars* sc, int renorm,
                            int advance, int finalize);
    static cudaError_t coef(cudaStream_t s, void* fa, void* fg, void* fp, void* fq, int n, double bre, double bim);
    static cudaError_t flush(cudaStream_t s, void* A, size_t plane, const DevScalars* sc);
    static cudaError_t norms(cudaStream_t s, const void* A, size_t plane, double cell, int renorm, double mag,
                             double* partials, DevScalars* sc);
    static cudaError_t observables(cudaStream_t s, const void* A, const KParams& p, double omega_t,
                                   double* partials, DevScalars* sc);
};

cudaError_t reset_scale(cudaStream_t s, DevScalars* sc);

// Store the message that sgpe_last_error(NULL) returns on this host thread.
void set_thread_error(const char* msg);

}  // namespace sgpe
