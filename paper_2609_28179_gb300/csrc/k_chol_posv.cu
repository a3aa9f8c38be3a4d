// k_chol_posv.cu -- instantiation unit of the batched posv kernels (one
// translation unit per operation keeps the parallel build short).
#include "k_chol_impl.cuh"

namespace glass {
cudaError_t launch_posv(int n, int nrhs, Mat A, Mat B, int *info, int batch, Placement pl, int num,
                        int refine, cudaStream_t st) {
    return run<C_POSV>(n, nrhs, A, B, info, batch, pl, num, refine, st);
}

// op: GLASS_OP_POTRF / POTRS / TRSM / POSV
size_t smem_chol(int op, int n, int nrhs, Placement pl) {
    switch (op) {
        case GLASS_OP_POTRF: return smem_of<C_POTRF>(n, nrhs, pl, 0);
        case GLASS_OP_POTRS: return smem_of<C_POTRS>(n, nrhs, pl, 0);
        case GLASS_OP_TRSM: return smem_of<C_TRSM>(n, nrhs, pl, 0);
        default: return smem_of<C_POSV>(n, nrhs, pl, 1);
    }
}

bool feasible_chol(int op, int n, int nrhs, Placement pl) {
    switch (op) {
        case GLASS_OP_POTRF: return feasible_of<C_POTRF>(n, nrhs, pl, 0);
        case GLASS_OP_POTRS: return feasible_of<C_POTRS>(n, nrhs, pl, 0);
        case GLASS_OP_TRSM: return feasible_of<C_TRSM>(n, nrhs, pl, 0);
        default: return feasible_of<C_POSV>(n, nrhs, pl, 0);
    }
}

}  // namespace glass
