#include "common.cuh"
namespace glass {
cudaError_t launch_gemm_tc(int, int, const void *, const void *, float *, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace glass
