#include "common.cuh"
namespace glass {
size_t varsize_workspace(int batch) { return 256 + (size_t)batch * 8; }
cudaError_t launch_posv_varsize(int, const int *, const long long *, const long long *, int, float *, float *, int *,
                                void *, int, unsigned *, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace glass
