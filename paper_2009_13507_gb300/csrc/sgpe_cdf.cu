// Double-float (FP32-pair) instantiation of the step, observable and COEF
// kernels: the FP64-accurate form computed on the FP32 pipe.
#include "sgpe_launch_impl.cuh"

namespace sgpe {
template struct Launcher<df>;

static __global__ void k_split_c128(const double2* __restrict__ src, float4* __restrict__ dst, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        dst[i] = pack(cx<df>{df_from(v.x), df_from(v.y)});
    }
}

cudaError_t cdf_from_c128(cudaStream_t s, const void* src, void* dst, size_t n) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_split_c128<<<(unsigned)blocks, 256, 0, s>>>((const double2*)src, (float4*)dst, n);
    return cudaGetLastError();
}
}  // namespace sgpe
