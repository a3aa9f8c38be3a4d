// k_varsize.cu -- fused SPD factor + solve over a batch of instances of
// different orders in one persistent launch (a batching pattern outside the
// paper; each instance runs the warp-scope posv primitive of Sec. III-A).
//
// 1. k_varsize_bin (one CTA): histogram of the orders, a descending scan
//    (largest orders first: longest-processing-time order, so the tail of
//    each launch is made of its cheapest instances), the scatter of the
//    instance indices into `order`, and the ranges of the four order
//    buckets (33..64, 17..32, 9..16, 1..8).  Instances with an order outside
//    [1, 64] get info = -1 and are left out.  The tickets are reset here.
// 2. k_varsize_posv<NMAX> (persistent, one launch per bucket, largest
//    first, grid = resident CTAs of that instantiation): every warp takes
//    the next ticket of its bucket with one atomic, solves instance
//    order[start + ticket] with the warp primitive specialised for the
//    bucket (the register-resident factorization up to order 16, the
//    blocked tensor-core one in the warp's shared memory above), and
//    repeats.  One instantiation per bucket keeps each launch at
//    the register count of its own order.  No CTA ever waits on another.
//
// Everything the launch needs lives in the caller's workspace, so the pair
// of kernels can be recorded in a CUDA graph and replayed.
#include "dev_chol.cuh"
#include "dev_chol_tc.cuh"

namespace glass {
namespace {

struct VarWs {
    int ticket[4];   // per bucket
    int bstart[4];   // bucket ranges in order[]
    int bcount[4];
    int valid;
    int pad[51];
    int count[65];
    int start[65];
    // followed by int order[batch]
};

// Bucket of an order: 0 -> 33..64, 1 -> 17..32, 2 -> 9..16, 3 -> 1..8.
__host__ __device__ __forceinline__ int bucket_of(int n) { return n > 32 ? 0 : n > 16 ? 1 : n > 8 ? 2 : 3; }

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
        for (int q = 0; q < 4; ++q) {
            const int hi = q == 0 ? 64 : q == 1 ? 32 : q == 2 ? 16 : 8;
            const int lo = q == 0 ? 33 : q == 1 ? 17 : q == 2 ? 9 : 1;
            int c = 0;
            for (int n = lo; n <= hi; ++n) c += cnt[n];
            ws->bstart[q] = cur[hi];
            ws->bcount[q] = c;
            ws->ticket[q] = 0;
        }
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
    for (int c = 0; c < nrhs; ++c) {
        float x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            x[q] = (i < n) ? __ldcs(B + c * n + i) : 0.f;
        }
        tcwarp::potrs<NMAX>(As, dv, x, n);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            if (i < n) __stcs(B + c * n + i, x[q]);
        }
    }
    tcwarp::unstage<NMAX, true>(A, n, As, n);
    return info;
}

// Shared-memory floats per warp of a bucket.
template <int NMAX>
constexpr int bucket_floats() {
    return NMAX >= 32 ? NMAX * (NMAX + 8) + NMAX + 32 : NMAX;
}

template <int NMAX>
__global__ void __launch_bounds__(256) k_varsize_posv(const int *__restrict__ n_dev, const long long *__restrict__ offA,
                                                      const long long *__restrict__ offB, int nrhs, float *A, float *B,
                                                      int *__restrict__ info, VarWs *ws, int bucket) {
    extern __shared__ __align__(16) float vsm[];
    const int lane = threadIdx.x & 31;
    float *col = vsm + (threadIdx.x >> 5) * bucket_floats<NMAX>();
    const int *order = reinterpret_cast<const int *>(ws + 1);
    const int start = ws->bstart[bucket], count = ws->bcount[bucket];
    // software pipeline: lane 0 takes the next ticket and fetches that
    // instance's metadata before the current instance is solved; the warp
    // reads them (shuffles) only afterwards, so their latency overlaps it
    int t = 0;
    if (lane == 0) t = atomicAdd(&ws->ticket[bucket], 1);
    t = __shfl_sync(GLASS_FULL_MASK, t, 0);
    int i = t < count ? order[start + t] : 0;
    int n = t < count ? n_dev[i] : 0;
    long long oa = t < count ? offA[i] : 0, ob = t < count ? offB[i] : 0;
    while (t < count) {
        int t2 = count, i2 = 0, n2 = 0;
        long long oa2 = 0, ob2 = 0;
        if (lane == 0) {
            t2 = atomicAdd(&ws->ticket[bucket], 1);
            if (t2 < count) {
                i2 = order[start + t2];
                n2 = n_dev[i2];
                oa2 = offA[i2];
                ob2 = offB[i2];
            }
        }
        int inf;
        if constexpr (NMAX >= 32) inf = warp_posv_tc<NMAX>(A + oa, B + ob, n, nrhs, col);
        else inf = warp_posv_one<NMAX>(A + oa, B + ob, n, nrhs, col);
        if (lane == 0) info[i] = inf;
        t = __shfl_sync(GLASS_FULL_MASK, t2, 0);
        i = __shfl_sync(GLASS_FULL_MASK, i2, 0);
        n = __shfl_sync(GLASS_FULL_MASK, n2, 0);
        oa = __shfl_sync(GLASS_FULL_MASK, oa2, 0);
        ob = __shfl_sync(GLASS_FULL_MASK, ob2, 0);
    }
}

template <int NMAX>
cudaError_t launch_bucket(int batch, const int *n_dev, const long long *offA, const long long *offB, int nrhs, float *A,
                          float *B, int *info, VarWs *w, int warps_per_cta, int bucket, int sms, cudaStream_t st) {
    const int threads = 32 * warps_per_cta;
    const size_t sm = (size_t)warps_per_cta * bucket_floats<NMAX>() * 4;
    cudaError_t pe = prepare_kernel(reinterpret_cast<const void *>(k_varsize_posv<NMAX>), sm);
    if (pe != cudaSuccess) return pe;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_varsize_posv<NMAX>, threads, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long want = (long long)sms * per_sm;
    const long long need = ((long long)batch + warps_per_cta - 1) / warps_per_cta;
    const int grid = (int)(want < need ? want : need);
    k_varsize_posv<NMAX><<<grid, threads, sm, st>>>(n_dev, offA, offB, nrhs, A, B, info, w, bucket);
    return cudaPeekAtLastError();
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
    if ((e = launch_bucket<64>(batch, n_dev, offA, offB, nrhs, A, B, info, w, warps_per_cta, 0, sms, st)) != cudaSuccess)
        return e;
    if ((e = launch_bucket<32>(batch, n_dev, offA, offB, nrhs, A, B, info, w, warps_per_cta, 1, sms, st)) != cudaSuccess)
        return e;
    if ((e = launch_bucket<16>(batch, n_dev, offA, offB, nrhs, A, B, info, w, warps_per_cta, 2, sms, st)) != cudaSuccess)
        return e;
    return launch_bucket<8>(batch, n_dev, offA, offB, nrhs, A, B, info, w, warps_per_cta, 3, sms, st);
}

}  // namespace glass
