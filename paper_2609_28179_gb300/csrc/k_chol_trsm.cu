// k_chol_trsm.cu -- instantiation unit of the batched trsm kernels (one
// translation unit per operation keeps the parallel build short).
#include "k_chol_impl.cuh"

namespace glass {
cudaError_t launch_trsm(int n, int nrhs, Mat L, Mat B, int batch, Placement pl, cudaStream_t st) {
    return run<C_TRSM>(n, nrhs, L, B, nullptr, batch, pl, 0, 0, st);
}

}  // namespace glass
