// k_varsize.cu -- fused SPD factor + solve over a batch of instances of
// different orders in one persistent launch (a batching pattern outside the
// paper; each instance runs the warp-scope posv primitive of Sec. III-A).
//
// 1. k_varsize_bin (one CTA): histogram of the orders, a descending scan
//    (largest orders first: longest-processing-time order, so the tail of
//    the launch is made of its cheapest instances) and the scatter of the
//    instance indices into `order`.  Instances with an order outside
//    [1, 64] get info = -1 and are left out.  The ticket is reset here.
// 2. k_varsize_posv (one persistent launch, grid = resident CTAs): every
//    warp takes the next ticket with one atomic and solves instance
//    order[ticket] with the warp primitive for its order -- the blocked
//    tensor-core Cholesky in the warp's shared memory above order 16 (64-
//    or 32-row variant), the register-resident one up to 16 -- and repeats
//    until the tickets run out.  All orders share the launch, so no order
//    class waits for the tail of another; no CTA ever waits on another.
//
// Everything the launch needs lives in the caller's workspace, so the pair
// of kernels can be recorded in a CUDA graph and replayed.
#include "dev_chol.cuh"
#include "dev_chol_tc.cuh"

namespace glass {
namespace {

struct VarWs {
    int ticket;     // next position of order[] to be taken
    int valid;      // instances with an order in [1, 64]
    int pad[62];
    int count[65];  // instances per order
    int start[65];  // first position of each order in order[]
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

// The same with the blocked tensor-core Cholesky (orders 17..NMAX, NMAX 32
// or 64) on the instance staged in the warp's shared memory As.
template <int NMAX>
__device__ __forceinline__ int warp_posv_tc(float *A, float *B, int n, int nrhs, float *As) {
    constexpr int LD = tcwarp::Shape<NMAX>::LD;
    constexpr int R = tcwarp::Shape<NMAX>::R;
    float *dv = As + NMAX * LD, *bc = dv + NMAX;
    const int lane = threadIdx.x & 31;
    __syncwarp();  // the previous instance is done with As
    tcwarp::stage<NMAX, true>(As, A, n, n);
    const int info = tcwarp::potrf<NMAX>(As, n, dv, bc, false);
    constexpr int K = 4;  // right-hand sides solved together (independent chains interleaved)
    for (int c0 = 0; c0 < nrhs; c0 += K) {
        float x[K][R];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                x[k][q] = (i < n && c0 + k < nrhs) ? __ldcs(B + (c0 + k) * n + i) : 0.f;
            }
        tcwarp::potrs_k<NMAX, K>(As, dv, x, n);
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (i < n && c0 + k < nrhs) __stcs(B + (c0 + k) * n + i, x[k][q]);
            }
    }
    tcwarp::unstage<NMAX, true>(A, n, As, n);
    return info;
}

// Shared-memory floats per warp: the 64-row tensor-core body's buffer
// (A at pitch 72, 1 / l_jj, 32 floats of broadcast scratch), which also
// holds every smaller body's.
constexpr int kWarpFloats = 64 * (64 + 8) + 64 + 32;

__global__ void __launch_bounds__(256) k_varsize_posv(const int *__restrict__ n_dev, const long long *__restrict__ offA,
                                                      const long long *__restrict__ offB, int nrhs, float *A, float *B,
                                                      int *__restrict__ info, VarWs *ws) {
    extern __shared__ __align__(16) float vsm[];
    const int lane = threadIdx.x & 31;
    float *col = vsm + (threadIdx.x >> 5) * kWarpFloats;
    const int *order = reinterpret_cast<const int *>(ws + 1);
    const int count = ws->valid;
    // software pipeline: lane 0 takes the next ticket and fetches that
    // instance's metadata before the current instance is solved; the warp
    // reads them (shuffles) only afterwards, so their latency overlaps it
    int t = 0;
    if (lane == 0) t = atomicAdd(&ws->ticket, 1);
    t = __shfl_sync(GLASS_FULL_MASK, t, 0);
    int i = t < count ? order[t] : 0;
    int n = t < count ? n_dev[i] : 0;
    long long oa = t < count ? offA[i] : 0, ob = t < count ? offB[i] : 0;
    while (t < count) {
        int t2 = count, i2 = 0, n2 = 0;
        long long oa2 = 0, ob2 = 0;
        if (lane == 0) {
            t2 = atomicAdd(&ws->ticket, 1);
            if (t2 < count) {
                i2 = order[t2];
                n2 = n_dev[i2];
                oa2 = offA[i2];
                ob2 = offB[i2];
            }
        }
        __syncwarp();  // every lane is done with the previous instance's shared memory
        int inf;  // the order is uniform over the warp, so is the branch
        if (n > 32) inf = warp_posv_tc<64>(A + oa, B + ob, n, nrhs, col);
        else if (n > 16) inf = warp_posv_tc<32>(A + oa, B + ob, n, nrhs, col);
        else if (n > 8) inf = warp_posv_one<16>(A + oa, B + ob, n, nrhs, col);
        else inf = warp_posv_one<8>(A + oa, B + ob, n, nrhs, col);
        if (lane == 0) info[i] = inf;
        t = __shfl_sync(GLASS_FULL_MASK, t2, 0);
        i = __shfl_sync(GLASS_FULL_MASK, i2, 0);
        n = __shfl_sync(GLASS_FULL_MASK, n2, 0);
        oa = __shfl_sync(GLASS_FULL_MASK, oa2, 0);
        ob = __shfl_sync(GLASS_FULL_MASK, ob2, 0);
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
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int threads = 32 * warps_per_cta;
    const size_t sm = (size_t)warps_per_cta * kWarpFloats * 4;
    if ((e = prepare_kernel(reinterpret_cast<const void *>(k_varsize_posv), sm)) != cudaSuccess) return e;
    int per_sm = 0;
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
