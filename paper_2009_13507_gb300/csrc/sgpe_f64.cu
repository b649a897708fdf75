// Complex128 (FP64) instantiation of the step, observable and COEF kernels.
#include "sgpe_launch_impl.cuh"

namespace sgpe {
template struct Launcher<double>;

cudaError_t reset_scale(cudaStream_t s, DevScalars* sc) {
    k_reset_scale<<<1, 32, 0, s>>>(sc);
    return cudaGetLastError();
}
}  // namespace sgpe
