// k_chol_impl.cuh -- batched potrf / potrs / trsm / posv kernels at thread, warp
// and block scope, plus the FP64-residual refinement step of posv.
//
// Each kernel wraps a device primitive of dev_chol.cuh with the batched
// load / compute / store of one placement (scope x pack, Sec. III-A).  Thread
// scope stages its 32*pack problems through shared memory with coalesced
// 16-byte streaming loads (column-major input) or reads the interleaved
// layout directly; warp scope loads rows straight into registers (each
// column of a problem is a contiguous, coalesced segment); block scope
// stages each problem into its team's shared memory.
#pragma once
#include "dev_chol.cuh"

namespace glass {
namespace {

enum CholOp { C_POTRF = 0, C_POTRS = 1, C_TRSM = 2, C_POSV = 3 };

constexpr bool has_factor(int op) { return op == C_POTRF || op == C_POSV; }
constexpr bool has_rhs(int op) { return op != C_POTRF; }

// r = b - A x in FP64 for one problem, A symmetric with its lower triangle
// read from `a` (column-major, leading dimension lda, ELEMENT accessor).
// Used by the refinement step: the factorization and first solve are FP32.

// ------------------------------------------------------------ thread scope
template <int OP, int NMAX, bool EXACT>
__global__ void __launch_bounds__(256) k_chol_thread(int n_rt, int nrhs, Mat A, Mat B, int *info,
                                                     int batch, int fp64diag, int refine) {
    extern __shared__ float smem[];
    using TR = Tri<NMAX>;
    const int n = EXACT ? NMAX : n_rt;
    const int G = blockDim.x;
    const int b0 = blockIdx.x * G;
    const int cnt = min(G, batch - b0);
    const int t = threadIdx.x;
    const bool staged = A.layout == GLASS_LAYOUT_COLMAJOR;
    const int SA = odd_stride(n * n);
    const int SB = has_rhs(OP) ? odd_stride(n * nrhs) : 0;
    float *sa = smem;
    float *sb = smem + G * SA;
    if (staged) {
        stage_in(sa, SA, A, b0, cnt);
        if (has_rhs(OP)) stage_in(sb, SB, B, b0, cnt);
        __syncthreads();
    }
    if (t < cnt) {
        const int b = b0 + t;
        const float *pa = sa + t * SA;
        float a[TR::size];
        float dinv[NMAX];
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
#pragma unroll
            for (int i = j; i < NMAX; ++i)
                a[TR::idx(i, j)] = (i < n) ? (staged ? pa[j * n + i] : A.get(b, i, j)) : 0.f;
        if (has_factor(OP)) {
            const int inf = thread::potrf<NMAX, EXACT>(a, dinv, n, fp64diag != 0);
            info[b] = inf;
        } else {
#pragma unroll
            for (int j = 0; j < NMAX; ++j) dinv[j] = (j < n) ? 1.0f / a[TR::idx(j, j)] : 0.f;
        }
        if (has_rhs(OP)) {
            float *pb = sb + t * SB;
            for (int c = 0; c < nrhs; ++c) {
                float x[NMAX];
#pragma unroll
                for (int i = 0; i < NMAX; ++i)
                    x[i] = (i < n) ? (staged ? pb[c * n + i] : B.get(b, i, c)) : 0.f;
                thread::forward<NMAX, EXACT>(a, dinv, x, n);
                if (OP != C_TRSM) thread::backward_t<NMAX, EXACT>(a, dinv, x, n);
                if (OP == C_POSV && refine) {
                    // r = b - A x0 in FP64 (A and b are still pristine in the
                    // staging buffers / in global memory).
                    float r[NMAX];
#pragma unroll
                    for (int i = 0; i < NMAX; ++i) {
                        if (i < n) {
                            double acc = staged ? (double)pb[c * n + i] : (double)B.get(b, i, c);
#pragma unroll
                            for (int k = 0; k < NMAX; ++k) {
                                if (k < n) {
                                    const float aik = (k <= i) ? (staged ? pa[k * n + i] : A.get(b, i, k))
                                                               : (staged ? pa[i * n + k] : A.get(b, k, i));
                                    acc = fma(-(double)aik, (double)x[k], acc);
                                }
                            }
                            r[i] = (float)acc;
                        } else {
                            r[i] = 0.f;
                        }
                    }
                    thread::forward<NMAX, EXACT>(a, dinv, r, n);
                    thread::backward_t<NMAX, EXACT>(a, dinv, r, n);
#pragma unroll
                    for (int i = 0; i < NMAX; ++i) x[i] += r[i];
                }
#pragma unroll
                for (int i = 0; i < NMAX; ++i)
                    if (i < n) {
                        if (staged) pb[c * n + i] = x[i];
                        else B.set(b, i, c, x[i]);
                    }
            }
        }
        if (has_factor(OP)) {
            float *wa = sa + t * SA;
#pragma unroll
            for (int j = 0; j < NMAX; ++j)
#pragma unroll
                for (int i = j; i < NMAX; ++i)
                    if (i < n) {
                        if (staged) wa[j * n + i] = a[TR::idx(i, j)];
                        else A.set(b, i, j, a[TR::idx(i, j)]);
                    }
        }
    }
    if (staged) {
        __syncthreads();
        if (has_factor(OP)) stage_out(sa, SA, A, b0, cnt);
        if (has_rhs(OP)) stage_out(sb, SB, B, b0, cnt);
    }
}

// -------------------------------------------------------------- warp scope
template <int OP, int NMAX>
__global__ void __launch_bounds__(256) k_chol_warp(int n, int nrhs, Mat A, Mat B, int *info, int batch,
                                                   int fp64diag, int refine) {
    constexpr int R = warp::Rows<NMAX>::R;
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;  // whole warp
    float a[R][NMAX];
    float rd[R];
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            a[q][k] = (k < n && i < n && k <= i) ? A.get(b, i, k) : 0.f;
        }
    if (has_factor(OP)) {
        const int inf = warp::potrf<NMAX>(a, rd, n, fp64diag != 0);
        if (lane == 0) info[b] = inf;
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            float dii = 1.f;
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k == i) dii = a[q][k];
            rd[q] = (i < n) ? 1.0f / dii : 0.f;
        }
    }
    if (has_rhs(OP)) {
        for (int c = 0; c < nrhs; ++c) {
            float x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                x[q] = (i < n) ? B.get(b, i, c) : 0.f;
            }
            warp::forward<NMAX>(a, rd, x, n);
            if (OP != C_TRSM) warp::backward_t<NMAX>(a, rd, x, n);
            if (OP == C_POSV && refine) {
                // r_i = b_i - sum_k a_ik x_k in FP64; A is re-read from
                // global memory (not yet overwritten: L is stored last).
                double acc[R];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int i = lane + 32 * q;
                    acc[q] = (i < n) ? (double)B.get(b, i, c) : 0.0;
                }
                for (int k = 0; k < n; ++k) {
                    float xk = 0.f;
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const float v = __shfl_sync(GLASS_FULL_MASK, x[q], k & 31);
                        if ((k >> 5) == q) xk = v;
                    }
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int i = lane + 32 * q;
                        if (i < n) {
                            const float aik = (k <= i) ? A.get(b, i, k) : A.get(b, k, i);
                            acc[q] = fma(-(double)aik, (double)xk, acc[q]);
                        }
                    }
                }
                float r[R];
#pragma unroll
                for (int q = 0; q < R; ++q) r[q] = (float)acc[q];
                warp::forward<NMAX>(a, rd, r, n);
                warp::backward_t<NMAX>(a, rd, r, n);
#pragma unroll
                for (int q = 0; q < R; ++q) x[q] += r[q];
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (i < n) B.set(b, i, c, x[q]);
            }
        }
    }
    if (has_factor(OP)) {
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (k < n && i < n && k <= i) A.set(b, i, k, a[q][k]);
            }
    }
}

// Warp-scope TRSM with many right-hand sides: L (and 1/l_ii) staged in the
// warp's shared memory, lane c solving column c (and c+32, ...).
template <int NMAX>
__global__ void __launch_bounds__(256) k_trsm_warp(int n, int nrhs, Mat L, Mat B, int batch) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int b = blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= batch) return;
    float *Ls = smem + w * (NMAX * NMAX + NMAX);
    float *dv = Ls + NMAX * NMAX;
    for (int e = lane; e < n * n; e += 32) {
        const int j = e / n, i = e - j * n;
        Ls[j * NMAX + i] = (i >= j) ? L.get(b, i, j) : 0.f;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) dv[i] = 1.0f / Ls[i * NMAX + i];
    __syncwarp();
    for (int c0 = 0; c0 < nrhs; c0 += 32) {
        const int c = c0 + lane;
        if (c < nrhs) {
            float x[NMAX];
#pragma unroll
            for (int i = 0; i < NMAX; ++i) x[i] = (i < n) ? B.get(b, i, c) : 0.f;
            warp::forward_cols<NMAX>(Ls, NMAX, dv, x, n);
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                if (i < n) B.set(b, i, c, x[i]);
        }
    }
}

// ------------------------------------------------------------- block scope
template <int OP, int T>
__global__ void __launch_bounds__(1024) k_chol_block(int n, int nrhs, Mat A, Mat B, int *info, int batch,
                                                    int fp64diag, int refine) {
    extern __shared__ float smem[];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const int P = blockDim.x / T;
    const int b = blockIdx.x * P + team;
    const int bar = 1 + team;
    const int lda = n | 1;
    const int per = n * lda + n + (has_rhs(OP) ? n * nrhs : 0) + ((OP == C_POSV && refine) ? 2 * n : 0);
    float *a = smem + team * per;
    float *dinv = a + n * lda;
    float *x = dinv + n;
    float *rr = x + (has_rhs(OP) ? n * nrhs : 0);
    if (b >= batch) return;  // the whole team leaves together
    for (int e = rank; e < n * n; e += T) {
        const int j = e / n, i = e - j * n;
        if (i >= j) a[j * lda + i] = A.get(b, i, j);
    }
    if (has_rhs(OP))
        for (int e = rank; e < n * nrhs; e += T) {
            const int c = e / n, i = e - c * n;
            x[c * n + i] = B.get(b, i, c);
        }
    team_sync<T>(bar);
    if (has_factor(OP)) {
        const int inf = block::potrf<T>(a, lda, n, rank, bar, fp64diag != 0, dinv);
        if (rank == 0) info[b] = inf;
    } else {
        block::diag_inverse<T>(a, lda, n, rank, bar, dinv);
    }
    if (has_rhs(OP)) {
        for (int c = 0; c < nrhs; ++c) {
            float *xc = x + c * n;
            block::forward<T>(a, lda, dinv, xc, n, rank, bar);
            if (OP != C_TRSM) block::backward_t<T>(a, lda, dinv, xc, n, rank, bar);
            if (OP == C_POSV && refine) {
                for (int i = rank; i < n; i += T) {
                    double acc = (double)B.get(b, i, c);
                    for (int k = 0; k < n; ++k) {
                        const float aik = (k <= i) ? A.get(b, i, k) : A.get(b, k, i);
                        acc = fma(-(double)aik, (double)xc[k], acc);
                    }
                    rr[i] = (float)acc;
                }
                team_sync<T>(bar);
                block::forward<T>(a, lda, dinv, rr, n, rank, bar);
                block::backward_t<T>(a, lda, dinv, rr, n, rank, bar);
                for (int i = rank; i < n; i += T) xc[i] += rr[i];
                team_sync<T>(bar);
            }
        }
        for (int e = rank; e < n * nrhs; e += T) {
            const int c = e / n, i = e - c * n;
            B.set(b, i, c, x[c * n + i]);
        }
    }
    if (has_factor(OP))
        for (int e = rank; e < n * n; e += T) {
            const int j = e / n, i = e - j * n;
            if (i >= j) A.set(b, i, j, a[j * lda + i]);
        }
}

// ---------------------------------------------------------------- dispatch
template <typename K>
cudaError_t launch_k(K kern, int grid, int threads, size_t smem, cudaStream_t st, int n, int nrhs,
                     const Mat &A, const Mat &B, int *info, int batch, int fp64diag, int refine) {
    {
        cudaError_t e = prepare(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, threads, smem, st>>>(n, nrhs, A, B, info, batch, fp64diag, refine);
    return cudaPeekAtLastError();
}

constexpr size_t kMaxSmem = 227 * 1024;

// Thread-scope instantiations: exact orders of the placement sweep and
// buckets (runtime order <= NMAX) for the rest.
template <int OP>
cudaError_t thread_dispatch(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, int pack,
                            int fp64diag, int refine, cudaStream_t st) {
    const int G = 32 * pack;
    const bool staged = A.layout == GLASS_LAYOUT_COLMAJOR;
    const size_t smem = staged ? (size_t)G * (odd_stride(n * n) + (has_rhs(OP) ? odd_stride(n * nrhs) : 0)) * 4 : 0;
    const int grid = ceil_div(batch, G);
#define GL_T(N, EX) launch_k(k_chol_thread<OP, N, EX>, grid, G, smem, st, n, nrhs, A, B, info, batch, fp64diag, refine)
    switch (n) {
        case 3: return GL_T(3, true);
        case 6: return GL_T(6, true);
        case 7: return GL_T(7, true);
        case 12: return GL_T(12, true);
        case 14: return GL_T(14, true);
        default: break;
    }
    if (n <= 2) return GL_T(2, false);
    if (n <= 4) return GL_T(4, false);
    if (n <= 8) return GL_T(8, false);
    if (n <= 12) return GL_T(12, false);
    if (n <= 16) return GL_T(16, false);
#undef GL_T
    return cudaErrorInvalidValue;
}

template <int OP>
cudaError_t warp_dispatch(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, int pack,
                          int fp64diag, int refine, cudaStream_t st) {
    const int threads = 32 * pack;
    const int grid = ceil_div(batch, pack);
    if (OP == C_TRSM) {
#define GL_TW(N) do { auto kern = k_trsm_warp<N>; size_t sm = (size_t)pack * (N * N + N) * 4;                 \
        { cudaError_t e = prepare(kern, sm); if (e != cudaSuccess) return e; }                                 \
        kern<<<grid, threads, sm, st>>>(n, nrhs, A, B, batch); return cudaPeekAtLastError(); } while (0)
        if (n <= 8) GL_TW(8);
        if (n <= 16) GL_TW(16);
        if (n <= 32) GL_TW(32);
        GL_TW(64);
#undef GL_TW
    }
#define GL_W(N) launch_k(k_chol_warp<OP, N>, grid, threads, 0, st, n, nrhs, A, B, info, batch, fp64diag, refine)
    if (n <= 8) return GL_W(8);
    if (n <= 16) return GL_W(16);
    if (n <= 32) return GL_W(32);
    return GL_W(64);
#undef GL_W
}

template <int OP>
size_t block_smem(int n, int nrhs, int pack, int refine) {
    const int lda = n | 1;
    const size_t per = (size_t)n * lda + n + (has_rhs(OP) ? (size_t)n * nrhs : 0) + ((OP == C_POSV && refine) ? 2 * n : 0);
    return per * pack * 4;
}

template <int OP>
cudaError_t block_dispatch(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, int pack,
                           int fp64diag, int refine, cudaStream_t st) {
    const int T = block_team(n);
    const size_t smem = block_smem<OP>(n, nrhs, pack, refine);
    const int grid = ceil_div(batch, pack);
    if (T == 64) return launch_k(k_chol_block<OP, 64>, grid, 64 * pack, smem, st, n, nrhs, A, B, info, batch, fp64diag, refine);
    if (T == 128) return launch_k(k_chol_block<OP, 128>, grid, 128 * pack, smem, st, n, nrhs, A, B, info, batch, fp64diag, refine);
    return launch_k(k_chol_block<OP, 256>, grid, 256 * pack, smem, st, n, nrhs, A, B, info, batch, fp64diag, refine);
}

template <int OP>
size_t smem_of(int n, int nrhs, Placement pl, int refine) {
    switch (pl.scope) {
        case SCOPE_THREAD:
            return (size_t)32 * pl.pack * (odd_stride(n * n) + (has_rhs(OP) ? odd_stride(n * nrhs) : 0)) * 4;
        case SCOPE_WARP: {
            if (OP != C_TRSM) return 0;
            const int N = n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64;
            return (size_t)pl.pack * (N * N + N) * 4;
        }
        default:
            return block_smem<OP>(n, nrhs, pl.pack, refine);
    }
}

template <int OP>
bool feasible_of(int n, int nrhs, Placement pl, int refine) {
    if (n < 1 || n > 64) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (pl.scope == SCOPE_THREAD && n > 16) return false;
    if (pl.scope == SCOPE_BLOCK && block_team(n) * pl.pack > 1024) return false;
    return smem_of<OP>(n, nrhs, pl, refine) <= kMaxSmem;
}

template <int OP>
cudaError_t run(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, Placement pl, int fp64diag,
                int refine, cudaStream_t st) {
    if (!feasible_of<OP>(n, nrhs, pl, refine)) return cudaErrorInvalidConfiguration;
    switch (pl.scope) {
        case SCOPE_THREAD: return thread_dispatch<OP>(n, nrhs, A, B, info, batch, pl.pack, fp64diag, refine, st);
        case SCOPE_WARP: return warp_dispatch<OP>(n, nrhs, A, B, info, batch, pl.pack, fp64diag, refine, st);
        default: return block_dispatch<OP>(n, nrhs, A, B, info, batch, pl.pack, fp64diag, refine, st);
    }
}

}  // namespace
}  // namespace glass
