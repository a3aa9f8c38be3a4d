#include "common.cuh"
namespace glass {
size_t mlp_workspace(int rows) { return 256 + (size_t)rows * 1024; }
cudaError_t launch_mlp_forward(int, const float *, int, const float *, float *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_mlp_loss_grad(int, const float *, int, const float *, const float *, const float *, float *, float *,
                                 void *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_mlp_adam(int, float *, const float *, float *, float *, int, float, float, float, float, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace glass
