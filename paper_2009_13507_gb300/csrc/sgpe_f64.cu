// Complex128 (FP64) instantiation of the step, observable and COEF kernels.
#include "sgpe_launch_impl.cuh"

namespace sgpe {
template struct Launcher<double>;

cudaError_t finalize_step(cudaStream_t s, const double* partials, int nblk, double cell, int renorm, double mag,
                          int advance, DevScalars* sc, int part_df) {
    if (nblk / 3 > 256)
        return launch_pdl(k_finalize_wide, dim3(1), dim3(96 * kFinWarps), 0, s, partials, nblk / 3, cell, renorm, mag,
                          advance, sc, part_df);
    return launch_pdl(k_finalize, dim3(1), dim3(96), 0, s, partials, nblk / 3, cell, renorm, mag, advance, sc,
                      part_df);
}

cudaError_t reset_scale(cudaStream_t s, DevScalars* sc) {
    k_reset_scale<<<1, 32, 0, s>>>(sc);
    return cudaGetLastError();
}
}  // namespace sgpe
