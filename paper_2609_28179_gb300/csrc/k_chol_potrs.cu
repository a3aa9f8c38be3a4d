// k_chol_potrs.cu -- instantiation unit of the batched potrs kernels (one
// translation unit per operation keeps the parallel build short).
#include "k_chol_impl.cuh"

namespace glass {
cudaError_t launch_potrs(int n, int nrhs, Mat L, Mat B, int batch, Placement pl, cudaStream_t st) {
    return run<C_POTRS>(n, nrhs, L, B, nullptr, batch, pl, 0, 0, st);
}

}  // namespace glass
