// sgpe_static.cu -- sgpe_observables_noalloc: the observables reduction of
// sgpe_energy for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs under a host framework which owns every device allocation through
// its own pool and forbids others, plug-ins that only receive pointers to the
// data they process, and latency-critical loops that must not pay for an
// allocation (or the synchronisation it can imply) at an arbitrary moment. For
// them this entry point keeps its scratch -- the per-block partial sums and the
// last-block ticket of the reduction -- in a file-scope device array that every
// GPU which loads the library holds until the process exits. The caller passes
// only the state (input) and a 16-double device buffer (output).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/sgpe.h"
#include "sgpe_kernels.cuh"
#include "sgpe_launch.h"

using namespace sgpe;

namespace {

// Scratch: a DevScalars block (tickets, error flag, observables) in the first
// 256 bytes, then the per-block partial sums (kObsAcc doubles per block).
constexpr size_t kScratchBytes = 1u << 20;  // 1 MiB per device
constexpr size_t kScalarsBytes = 256;
constexpr size_t kMaxBlocks = (kScratchBytes - kScalarsBytes) / (kObsAcc * sizeof(double));
static_assert(sizeof(DevScalars) <= kScalarsBytes, "DevScalars must fit its slot");

static __device__ __align__(256) unsigned char g_obs_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_obs_scratch on the current device, looked up once per
// device (in host code the symbol is only a host-side stand-in).
cudaError_t scratch_on_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_obs_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sgpe_status sgpe_observables_noalloc(const void* psi_dev, int dim, int nx, int ny, double dx, double dy,
                                                sgpe_precision prec, const sgpe_params* p, double* obs_dev,
                                                void* cuda_stream) {
    if (!psi_dev || !obs_dev || !p) {
        set_thread_error("sgpe_observables_noalloc: null pointer");
        return SGPE_EINVAL;
    }
    if (dim != 1 && dim != 2) {
        set_thread_error("sgpe_observables_noalloc: dim must be 1 or 2");
        return SGPE_EINVAL;
    }
    if (dim == 1) {
        ny = 1;
        dy = dx;
    }
    if (nx < 3 || (dim == 2 && ny < 3) || !(dx > 0.0) || !(dy > 0.0) || !isfinite(dx) || !isfinite(dy) ||
        (prec != SGPE_C128 && prec != SGPE_C64 && prec != SGPE_CDF) || p->so_type < 0 || p->so_type > 3 || !isfinite(p->c0) ||
        !isfinite(p->c2) || !isfinite(p->gamma) || !isfinite(p->omega) || !isfinite(p->wx) || !isfinite(p->wy)) {
        set_thread_error("sgpe_observables_noalloc: invalid grid or parameters");
        return SGPE_EINVAL;
    }
    if (((uintptr_t)psi_dev & 15) != 0 || ((uintptr_t)obs_dev & 7) != 0) {
        set_thread_error("sgpe_observables_noalloc: psi must be 16-byte and obs 8-byte aligned");
        return SGPE_EINVAL;
    }
    const size_t blocks = (size_t)ceil_div(nx, 32) * (size_t)ceil_div(ny, 4);
    if (blocks > kMaxBlocks) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "sgpe_observables_noalloc: grid %dx%d needs %zu reduction blocks, the static scratch holds %zu "
                 "(at most about %zu grid points)",
                 nx, ny, blocks, kMaxBlocks, kMaxBlocks * 128);
        set_thread_error(msg);
        return SGPE_EUNSUPPORTED;
    }
    unsigned char* base = nullptr;
    cudaError_t e = scratch_on_current_device(&base);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the same kernel constants as a context's sgpe_energy (dt plays no part in the observables)
    const KParams k = make_kparams(dim, nx, ny, dx, dy, p);
    DevScalars* sc = (DevScalars*)base;
    double* partials = (double*)(base + kScalarsBytes);
    // The scratch keeps the previous call's contents: the ticket and the error
    // flag must start at zero.
    if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), s);
    if (e == cudaSuccess)
        e = prec == SGPE_C128  ? Launcher<double>::observables(s, psi_dev, k, k.omega_t, partials, sc)
            : prec == SGPE_C64 ? Launcher<float>::observables(s, psi_dev, k, k.omega_t, partials, sc)
                               : Launcher<df>::observables(s, psi_dev, k, k.omega_t, partials, sc);
    if (e == cudaSuccess) e = cudaMemcpyAsync(obs_dev, sc->obs, SGPE_NOBS * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "sgpe_observables_noalloc: %s", cudaGetErrorString(e));
        set_thread_error(msg);
        return SGPE_ECUDA;
    }
    return SGPE_OK;
}
