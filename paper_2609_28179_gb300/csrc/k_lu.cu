// k_lu.cu -- batched getrf + getrs (partial pivoting) at thread, warp and
// block scope.  The batched wrappers follow k_chol.cu: thread scope stages
// 32*pack problems through shared memory, warp scope loads rows straight
// into registers, block scope keeps each problem in its team's shared
// memory.
#include "dev_lu.cuh"

namespace glass {
namespace {

template <int NMAX, bool EXACT>
__global__ void __launch_bounds__(256) k_lu_thread(int n_rt, int nrhs, Mat A, int *ipiv, Mat B, int *info,
                                                   int batch) {
    extern __shared__ float smem[];
    const int n = EXACT ? NMAX : n_rt;
    const int G = blockDim.x;
    const int b0 = blockIdx.x * G;
    const int cnt = min(G, batch - b0);
    const int t = threadIdx.x;
    const bool staged = A.layout == GLASS_LAYOUT_COLMAJOR;
    const int SA = odd_stride(n * n);
    const int SB = nrhs > 0 ? odd_stride(n * nrhs) : 0;
    float *sa = smem;
    float *sb = smem + G * SA;
    if (staged) {
        stage_in(sa, SA, A, b0, cnt);
        if (nrhs > 0) stage_in(sb, SB, B, b0, cnt);
        __syncthreads();
    }
    if (t < cnt) {
        const int b = b0 + t;
        float *pa = sa + t * SA;
        float a[NMAX][NMAX];
        int piv[NMAX];
        float rinv[NMAX];
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                a[i][j] = (i < n && j < n) ? (staged ? pa[j * n + i] : A.get(b, i, j)) : 0.f;
        info[b] = thread::getrf<NMAX, EXACT>(a, piv, rinv, n);
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
            if (j < n) ipiv[(long long)b * n + j] = piv[j];
        float *pb = sb + t * SB;
        for (int c = 0; c < nrhs; ++c) {
            float x[NMAX];
#pragma unroll
            for (int i = 0; i < NMAX; ++i) x[i] = (i < n) ? (staged ? pb[c * n + i] : B.get(b, i, c)) : 0.f;
            thread::getrs<NMAX, EXACT>(a, piv, rinv, x, n);
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                if (i < n) {
                    if (staged) pb[c * n + i] = x[i];
                    else B.set(b, i, c, x[i]);
                }
        }
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                if (i < n && j < n) {
                    if (staged) pa[j * n + i] = a[i][j];
                    else A.set(b, i, j, a[i][j]);
                }
    }
    if (staged) {
        __syncthreads();
        stage_out(sa, SA, A, b0, cnt);
        if (nrhs > 0) stage_out(sb, SB, B, b0, cnt);
    }
}

template <int NMAX>
__global__ void __launch_bounds__(256) k_lu_warp(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch) {
    constexpr int R = warp::LU<NMAX>::R;
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;
    float a[R][NMAX];
    int pos[R];
    int pp[NMAX];
    float prc[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            a[q][k] = (k < n && i < n) ? A.get(b, i, k) : 0.f;
        }
    const int inf = warp::getrf<NMAX>(a, pos, pp, prc, ipiv + (long long)b * n, n);
    if (lane == 0) info[b] = inf;
    for (int c = 0; c < nrhs; ++c) {
        float x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            x[q] = (i < n) ? B.get(b, i, c) : 0.f;
        }
        warp::getrs<NMAX>(a, pos, pp, prc, x, n);
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (lane + 32 * q < n) B.set(b, pos[q], c, x[q]);
    }
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (k < n && lane + 32 * q < n) A.set(b, pos[q], k, a[q][k]);
}

template <int T>
__global__ void __launch_bounds__(1024) k_lu_block(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch) {
    extern __shared__ float smem[];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const int P = blockDim.x / T;
    const int b = blockIdx.x * P + team;
    const int bar = 1 + team;
    const int lda = n | 1;
    const int per = n * lda + 2 * n + n * nrhs + 4;
    float *a = smem + team * per;
    int *piv = reinterpret_cast<int *>(a + n * lda);
    float *rinv = a + n * lda + n;
    float *x = rinv + n;
    float *sc = x + n * nrhs;
    if (b >= batch) return;
    for (int e = rank; e < n * n; e += T) {
        const int j = e / n, i = e - j * n;
        a[j * lda + i] = A.get(b, i, j);
    }
    for (int e = rank; e < n * nrhs; e += T) {
        const int c = e / n, i = e - c * n;
        x[c * n + i] = B.get(b, i, c);
    }
    team_sync<T>(bar);
    const int inf = block::getrf<T>(a, lda, n, piv, rinv, rank, bar, sc);
    if (rank == 0) info[b] = inf;
    for (int j = rank; j < n; j += T) ipiv[(long long)b * n + j] = piv[j];
    for (int c = 0; c < nrhs; ++c) block::getrs<T>(a, lda, piv, rinv, x + c * n, n, rank, bar);
    for (int e = rank; e < n * nrhs; e += T) {
        const int c = e / n, i = e - c * n;
        B.set(b, i, c, x[c * n + i]);
    }
    for (int e = rank; e < n * n; e += T) {
        const int j = e / n, i = e - j * n;
        A.set(b, i, j, a[j * lda + i]);
    }
}

template <typename K>
cudaError_t go(K kern, int grid, int threads, size_t smem, cudaStream_t st, int n, int nrhs, const Mat &A, int *ipiv,
               const Mat &B, int *info, int batch) {
    {
        cudaError_t e = prepare(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, threads, smem, st>>>(n, nrhs, A, ipiv, B, info, batch);
    return cudaPeekAtLastError();
}

constexpr size_t kMaxSmem = 227 * 1024;

size_t smem_lu(int n, int nrhs, Placement pl) {
    switch (pl.scope) {
        case SCOPE_THREAD: return (size_t)32 * pl.pack * (odd_stride(n * n) + (nrhs > 0 ? odd_stride(n * nrhs) : 0)) * 4;
        case SCOPE_WARP: return 0;
        default: return (size_t)pl.pack * (n * (n | 1) + 2 * n + n * nrhs + 4) * 4;
    }
}

}  // namespace

bool feasible_lu(int n, int nrhs, Placement pl) {
    if (n < 1 || n > 64 || nrhs < 0) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (pl.scope == SCOPE_THREAD && n > 12) return false;
    if (pl.scope == SCOPE_BLOCK && block_team(n) * pl.pack > 1024) return false;
    return smem_lu(n, nrhs, pl) <= kMaxSmem;
}

cudaError_t launch_getrf_getrs(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch, Placement pl,
                               cudaStream_t st) {
    if (!feasible_lu(n, nrhs, pl)) return cudaErrorInvalidConfiguration;
    const size_t smem = smem_lu(n, nrhs, pl);
    if (pl.scope == SCOPE_THREAD) {
        const int G = 32 * pl.pack;
        const int grid = ceil_div(batch, G);
        const size_t sm = A.layout == GLASS_LAYOUT_COLMAJOR ? smem : 0;
#define GL_T(N, EX) go(k_lu_thread<N, EX>, grid, G, sm, st, n, nrhs, A, ipiv, B, info, batch)
        switch (n) {
            case 3: return GL_T(3, true);
            case 6: return GL_T(6, true);
            case 7: return GL_T(7, true);
            case 12: return GL_T(12, true);
            default: break;
        }
        if (n <= 2) return GL_T(2, false);
        if (n <= 4) return GL_T(4, false);
        if (n <= 8) return GL_T(8, false);
        return GL_T(12, false);
#undef GL_T
    }
    const int grid = ceil_div(batch, pl.pack);
    if (pl.scope == SCOPE_WARP) {
        const int th = 32 * pl.pack;
        if (n <= 8) return go(k_lu_warp<8>, grid, th, 0, st, n, nrhs, A, ipiv, B, info, batch);
        if (n <= 16) return go(k_lu_warp<16>, grid, th, 0, st, n, nrhs, A, ipiv, B, info, batch);
        if (n <= 32) return go(k_lu_warp<32>, grid, th, 0, st, n, nrhs, A, ipiv, B, info, batch);
        return go(k_lu_warp<64>, grid, th, 0, st, n, nrhs, A, ipiv, B, info, batch);
    }
    const int T = block_team(n);
    if (T == 64) return go(k_lu_block<64>, grid, 64 * pl.pack, smem, st, n, nrhs, A, ipiv, B, info, batch);
    if (T == 128) return go(k_lu_block<128>, grid, 128 * pl.pack, smem, st, n, nrhs, A, ipiv, B, info, batch);
    return go(k_lu_block<256>, grid, 256 * pl.pack, smem, st, n, nrhs, A, ipiv, B, info, batch);
}

}  // namespace glass
