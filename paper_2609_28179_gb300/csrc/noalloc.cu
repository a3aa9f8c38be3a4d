// noalloc.cu -- glass_posv_varsize_noalloc: the mixed-size batched SPD
// solve for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a real-time control loop that forbids
// any allocation once it is running (an allocation can block on the driver
// and break its cycle deadline), or a host program whose device memory is
// owned by another allocator that must not be bypassed.  glass_posv_varsize
// asks its caller for scratch; this entry point instead keeps that scratch
// in a fixed array in the library's device image, sized for at most
// kNoallocMaxBatch instances.  The caller still passes inputs and outputs.
//
// The array is one per device and is shared by every call on that device:
// calls that overlap on the GPU (different streams, no ordering between
// them) race on it.  Each call rewrites all of the scratch it reads (the
// binning kernel resets the ticket and rebuilds the counts and the order),
// so nothing left over from an earlier call is ever used.
#include "common.cuh"

namespace glass {
namespace {

constexpr int kNoallocMaxBatch = 65536;

// Scratch of the mixed-size solve for kNoallocMaxBatch instances (the
// binning header plus one int per instance), held by every GPU that loads
// the library until the process exits.
constexpr size_t kNoallocBytes = 4096 + (size_t)kNoallocMaxBatch * sizeof(int);
static __device__ __align__(256) unsigned char g_varsize_scratch[kNoallocBytes];

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the kernels must be given
// this address.  It is looked up on every call rather than cached: a caller
// that destroys its context (cudaDeviceReset) gets the module loaded again,
// possibly at another address, and a cached pointer would then dangle.
cudaError_t scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_varsize_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace glass

extern "C" glass_status glass_posv_varsize_noalloc(int batch, const int *n_dev, const long long *offA_dev,
                                                   const long long *offB_dev, int nrhs, void *A, void *B, int *info,
                                                   const glass_opts *opts, glass_stream_t stream) {
    if (batch > glass::kNoallocMaxBatch) return GLASS_ERR_UNSUPPORTED;
    if (batch <= 0) return batch == 0 ? GLASS_OK : GLASS_ERR_INVALID_VALUE;
    const size_t need = glass_posv_varsize_workspace(batch);
    if (need > glass::kNoallocBytes) return GLASS_ERR_UNSUPPORTED;
    void *ws = nullptr;
    if (glass::scratch_address(&ws) != cudaSuccess) return GLASS_ERR_CUDA;
    return glass_posv_varsize(batch, n_dev, offA_dev, offB_dev, nrhs, A, B, info, ws, need, opts, stream);
}
