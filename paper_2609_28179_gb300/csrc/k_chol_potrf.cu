// k_chol_potrf.cu -- instantiation unit of the batched potrf kernels (one
// translation unit per operation keeps the parallel build short).
#include "k_chol_impl.cuh"

namespace glass {
cudaError_t launch_potrf(int n, Mat A, int *info, int batch, Placement pl, int num, cudaStream_t st) {
    Mat none = A;
    return run<C_POTRF>(n, 0, A, none, info, batch, pl, num, 0, st);
}

}  // namespace glass
