// Complex64 (FP32 state, FP64 reductions) instantiation of the step,
// observable and COEF kernels (the precision form).
#include "sgpe_launch_impl.cuh"

namespace sgpe {
template struct Launcher<float>;
}  // namespace sgpe
