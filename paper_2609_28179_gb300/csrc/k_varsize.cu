// k_varsize.cu -- fused SPD factor + solve over a batch of instances of
// different orders in one persistent launch (a batching pattern outside the
// paper; each instance runs the warp-scope posv primitive of Sec. III-A).
//
// 1. k_varsize_bin (one CTA): histogram of the orders, a descending scan
//    (largest orders first: longest-processing-time order, so the tail of
//    the launch is made of the cheapest instances), and the scatter of the
//    instance indices into `order`.  Instances with an order outside
//    [1, 64] get info = -1 and are left out.  The ticket is reset here.
// 2. k_varsize_posv (persistent, grid = resident CTAs): every warp takes the
//    next ticket with one atomic, solves instance order[ticket] with the
//    warp primitive of the bucket its order falls in, and repeats.  No CTA
//    ever waits on another.
//
// Everything the launch needs lives in the caller's workspace, so the pair
// of kernels can be recorded in a CUDA graph and replayed.
#include "dev_chol.cuh"

namespace glass {
namespace {

struct VarWs {
    int ticket;
    int valid;
    int pad[62];
    int count[65];
    int start[65];
    // followed by int order[batch]
};

__global__ void __launch_bounds__(1024) k_varsize_bin(int batch, const int *__restrict__ n_dev, int *__restrict__ info,
                                                      VarWs *ws) {
    __shared__ int cnt[65];
    __shared__ int cur[65];
    int *order = reinterpret_cast<int *>(ws + 1);
    for (int i = threadIdx.x; i < 65; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < batch; i += blockDim.x) {
        const int n = n_dev[i];
        if (n >= 1 && n <= 64) atomicAdd(&cnt[n], 1);
        else info[i] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int n = 64; n >= 1; --n) {  // descending: largest orders first
            cur[n] = s;
            ws->start[n] = s;
            ws->count[n] = cnt[n];
            s += cnt[n];
        }
        ws->valid = s;
        ws->ticket = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < batch; i += blockDim.x) {
        const int n = n_dev[i];
        if (n >= 1 && n <= 64) order[atomicAdd(&cur[n], 1)] = i;
    }
}

// One SPD system of order n <= NMAX solved by the calling warp (A lda = n,
// B ldb = n), LAPACK semantics: A <- L (lower), B <- X, returns info.
template <int NMAX>
__device__ __forceinline__ int warp_posv_one(float *A, float *B, int n, int nrhs, float *col) {
    constexpr int R = warp::Rows<NMAX>::R;
    const int lane = threadIdx.x & 31;
    float a[R][NMAX];
    float rd[R];
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            a[q][k] = (k < n && i < n && k <= i) ? __ldcs(A + k * n + i) : 0.f;
        }
    const int info = warp::potrf<NMAX>(a, rd, n, false, col);
    for (int c = 0; c < nrhs; ++c) {
        float x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            x[q] = (i < n) ? __ldcs(B + c * n + i) : 0.f;
        }
        warp::forward<NMAX>(a, rd, x, n);
        warp::backward_t<NMAX>(a, rd, x, n);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            if (i < n) __stcs(B + c * n + i, x[q]);
        }
    }
    float *wa = opaque(A);
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            if (k < n && i < n && k <= i) __stcs(wa + k * n + i, a[q][k]);
        }
    return info;
}

__global__ void __launch_bounds__(256) k_varsize_posv(const int *__restrict__ n_dev, const long long *__restrict__ offA,
                                                      const long long *__restrict__ offB, int nrhs, float *A, float *B,
                                                      int *__restrict__ info, VarWs *ws) {
    extern __shared__ __align__(16) float vsm[];
    const int lane = threadIdx.x & 31;
    float *col = vsm + (threadIdx.x >> 5) * 64;
    const int *order = reinterpret_cast<const int *>(ws + 1);
    const int valid = ws->valid;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&ws->ticket, 1);
        t = __shfl_sync(GLASS_FULL_MASK, t, 0);
        if (t >= valid) break;
        const int i = order[t];
        const int n = n_dev[i];
        float *a = A + offA[i];
        float *b = B + offB[i];
        int inf;
        if (n <= 8) inf = warp_posv_one<8>(a, b, n, nrhs, col);
        else if (n <= 16) inf = warp_posv_one<16>(a, b, n, nrhs, col);
        else if (n <= 32) inf = warp_posv_one<32>(a, b, n, nrhs, col);
        else inf = warp_posv_one<64>(a, b, n, nrhs, col);
        if (lane == 0) info[i] = inf;
    }
}

}  // namespace

size_t varsize_workspace(int batch) {
    const size_t bytes = sizeof(VarWs) + (size_t)(batch > 0 ? batch : 0) * sizeof(int);
    return (bytes + 255) / 256 * 256;
}

cudaError_t launch_posv_varsize(int batch, const int *n_dev, const long long *offA, const long long *offB, int nrhs,
                                float *A, float *B, int *info, void *ws, int warps_per_cta, unsigned *status,
                                cudaStream_t st) {
    (void)status;
    VarWs *w = static_cast<VarWs *>(ws);
    k_varsize_bin<<<1, 1024, 0, st>>>(batch, n_dev, info, w);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int threads = 32 * warps_per_cta;
    const size_t sm = (size_t)warps_per_cta * 64 * 4;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_varsize_posv, threads, sm)) != cudaSuccess)
        return e;
    if (per_sm < 1) per_sm = 1;
    const long long want = (long long)sms * per_sm;
    const long long need = ((long long)batch + warps_per_cta - 1) / warps_per_cta;
    const int grid = (int)(want < need ? want : need);
    k_varsize_posv<<<grid, threads, sm, st>>>(n_dev, offA, offB, nrhs, A, B, info, w);
    return cudaPeekAtLastError();
}

}  // namespace glass
