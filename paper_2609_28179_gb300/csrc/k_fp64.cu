// k_fp64.cu -- FP64 storage variants of the matrix operations (the paper's
// fp32 + fp64 sweep design, Sec. IV-A): GEMM, POTRF / POTRS / POSV, TRSM and
// GETRF + GETRS on column-major double operands, at thread scope (one
// problem per thread, operand in registers, n <= 8) and warp scope (one
// problem per warp, the matrix in shared memory, n <= 64).  The arithmetic
// follows the FP32 kernels' definitions (lower Cholesky with LAPACK info;
// partial pivoting, largest magnitude with the smallest row on ties,
// sequential-interchange ipiv); divisions are true divisions.  GB300's FP64
// pipe is narrow (about 1 TFLOP/s measured), so these kernels aim at a
// correct, placement-measurable path rather than the FP32 kernels' depth.
#include "common.cuh"

namespace glass {
namespace {

constexpr int kF64MaxThreadN = 8;

// ----------------------------------------------------------------- GEMM
template <int NMAX>
__global__ void __launch_bounds__(256) k_gemm_f64_thread(int m, int n, int k, const double *A, int lda, long long sA,
                                                         const double *B, int ldb, long long sB, double *C, int ldc,
                                                         long long sC, int batch) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const double *a = A + b * sA, *bb = B + b * sB;
    double *c = C + b * sC;
    double ar[NMAX][NMAX];
#pragma unroll
    for (int l = 0; l < NMAX; ++l)
#pragma unroll
        for (int i = 0; i < NMAX; ++i) ar[i][l] = (i < m && l < k) ? a[(long long)l * lda + i] : 0.0;
    for (int j = 0; j < n; ++j) {
        double bc[NMAX];
#pragma unroll
        for (int l = 0; l < NMAX; ++l) bc[l] = l < k ? bb[(long long)j * ldb + l] : 0.0;
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < NMAX; ++l) s = fma(ar[i][l], bc[l], s);
            if (i < m) c[(long long)j * ldc + i] = s;
        }
    }
}

__global__ void __launch_bounds__(256) k_gemm_f64_warp(int m, int n, int k, const double *A, int lda, long long sA,
                                                       const double *B, int ldb, long long sB, double *C, int ldc,
                                                       long long sC, int batch) {
    const int lane = threadIdx.x & 31;
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;
    const double *a = A + b * sA, *bb = B + b * sB;
    double *c = C + b * sC;
    for (int j = 0; j < n; ++j) {
        double s0 = 0.0, s1 = 0.0;
        for (int l = 0; l < k; ++l) {
            const double blj = bb[(long long)j * ldb + l];
            if (lane < m) s0 = fma(a[(long long)l * lda + lane], blj, s0);
            if (lane + 32 < m) s1 = fma(a[(long long)l * lda + lane + 32], blj, s1);
        }
        if (lane < m) c[(long long)j * ldc + lane] = s0;
        if (lane + 32 < m) c[(long long)j * ldc + lane + 32] = s1;
    }
}

// ------------------------------------------------------- thread-scope solves
// OP: 0 potrf, 1 potrs, 2 posv, 3 trsm (C_* order of the FP32 kernels).
template <int OP, int NMAX>
__global__ void __launch_bounds__(256) k_chol_f64_thread(int n, int nrhs, double *A, int lda, long long sA, double *B,
                                                         int ldb, long long sB, int *info, int batch) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    double *a = A + b * sA;
    double L[NMAX][NMAX];
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
#pragma unroll
        for (int i = 0; i < NMAX; ++i) L[i][j] = (i < n && j < n && i >= j) ? a[(long long)j * lda + i] : 0.0;
    int inf = 0;
    if (OP == 0 || OP == 2) {
#pragma unroll
        for (int j = 0; j < NMAX; ++j) {
            if (j < n) {
                const double d = L[j][j];
                if (!(d > 0.0) && inf == 0) inf = j + 1;
                const double l = sqrt(d);
                L[j][j] = l;
#pragma unroll
                for (int i = j + 1; i < NMAX; ++i) L[i][j] = L[i][j] / l;
#pragma unroll
                for (int kk = j + 1; kk < NMAX; ++kk)
#pragma unroll
                    for (int i = kk; i < NMAX; ++i) L[i][kk] = fma(-L[i][j], L[kk][j], L[i][kk]);
            }
        }
        info[b] = inf;
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                if (i < n && j < n && i >= j) a[(long long)j * lda + i] = L[i][j];
    }
    if (OP == 0) return;
    double *bb = B + b * sB;
    for (int c = 0; c < nrhs; ++c) {
        double x[NMAX];
#pragma unroll
        for (int i = 0; i < NMAX; ++i) x[i] = i < n ? bb[(long long)c * ldb + i] : 0.0;
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            if (i < n) {
                double s = x[i];
#pragma unroll
                for (int kk = 0; kk < i; ++kk) s = fma(-L[i][kk], x[kk], s);
                x[i] = s / L[i][i];
            }
        }
        if (OP != 3) {
#pragma unroll
            for (int i = NMAX - 1; i >= 0; --i) {
                if (i < n) {
                    double s = x[i];
#pragma unroll
                    for (int kk = i + 1; kk < NMAX; ++kk) s = fma(-L[kk][i], x[kk], s);
                    x[i] = s / L[i][i];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
            if (i < n) bb[(long long)c * ldb + i] = x[i];
    }
}

template <int NMAX>
__global__ void __launch_bounds__(256) k_lu_f64_thread(int n, int nrhs, double *A, int lda, long long sA, int *ipiv,
                                                       double *B, int ldb, long long sB, int *info, int batch) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    double *a = A + b * sA;
    double M[NMAX][NMAX];
    int piv[NMAX];
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
#pragma unroll
        for (int i = 0; i < NMAX; ++i) M[i][j] = (i < n && j < n) ? a[(long long)j * lda + i] : 0.0;
    int inf = 0;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            int p = j;
            double best = fabs(M[j][j]);
#pragma unroll
            for (int i = j + 1; i < NMAX; ++i)
                if (i < n && fabs(M[i][j]) > best) { best = fabs(M[i][j]); p = i; }
            piv[j] = p;
            // interchange rows j and p (select chains: p is a run-time index)
#pragma unroll
            for (int c = 0; c < NMAX; ++c) {
                double rp = M[j][c];
#pragma unroll
                for (int i = j + 1; i < NMAX; ++i)
                    if (i == p) rp = M[i][c];
#pragma unroll
                for (int i = j + 1; i < NMAX; ++i)
                    if (i == p) M[i][c] = M[j][c];
                M[j][c] = rp;
            }
            const double pv = M[j][j];
            if (pv == 0.0) {
                if (inf == 0) inf = j + 1;
            } else {
#pragma unroll
                for (int i = j + 1; i < NMAX; ++i) M[i][j] = M[i][j] / pv;
#pragma unroll
                for (int c = j + 1; c < NMAX; ++c)
#pragma unroll
                    for (int i = j + 1; i < NMAX; ++i) M[i][c] = fma(-M[i][j], M[j][c], M[i][c]);
            }
        }
    }
    info[b] = inf;
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
        if (j < n) ipiv[b * n + j] = piv[j];
    double *bb = B + b * sB;
    for (int c = 0; c < nrhs; ++c) {
        double x[NMAX];
#pragma unroll
        for (int i = 0; i < NMAX; ++i) x[i] = i < n ? bb[(long long)c * ldb + i] : 0.0;
#pragma unroll
        for (int j = 0; j < NMAX; ++j) {  // the interchanges in order
            if (j < n) {
                double xp = x[j];
#pragma unroll
                for (int i = j + 1; i < NMAX; ++i)
                    if (i == piv[j]) xp = x[i];
#pragma unroll
                for (int i = j + 1; i < NMAX; ++i)
                    if (i == piv[j]) x[i] = x[j];
                x[j] = xp;
            }
        }
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            double s = x[i];
#pragma unroll
            for (int kk = 0; kk < i; ++kk) s = fma(-M[i][kk], x[kk], s);
            x[i] = s;
        }
#pragma unroll
        for (int i = NMAX - 1; i >= 0; --i) {
            if (i < n) {
                double s = x[i];
#pragma unroll
                for (int kk = i + 1; kk < NMAX; ++kk) s = fma(-M[i][kk], x[kk], s);
                x[i] = s / M[i][i];
            }
        }
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
            if (i < n) bb[(long long)c * ldb + i] = x[i];
    }
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
            if (i < n && j < n) a[(long long)j * lda + i] = M[i][j];
}

// --------------------------------------------------------- warp-scope solves
// The matrix lives in the warp's shared memory (column-major, odd pitch P);
// every step is lanes over rows (or columns) with a __syncwarp between steps.
__device__ __forceinline__ void stage_f64(double *S, int P, const double *g, int lda, int n, int lane, bool lower) {
    for (int e = lane; e < n * n; e += 32) {
        const int j = e / n, i = e - j * n;
        S[j * P + i] = (!lower || i >= j) ? g[(long long)j * lda + i] : 0.0;
    }
    __syncwarp();
}

__device__ __forceinline__ int potrf_f64_warp(double *S, int P, int n, int lane) {
    int inf = 0;
    for (int j = 0; j < n; ++j) {
        const double d = S[j * P + j];
        if (!(d > 0.0) && inf == 0) inf = j + 1;
        const double l = sqrt(d);
        __syncwarp();
        if (lane == 0) S[j * P + j] = l;
        for (int i = j + 1 + lane; i < n; i += 32) S[j * P + i] = S[j * P + i] / l;
        __syncwarp();
        for (int kk = j + 1; kk < n; ++kk) {
            const double lkj = S[j * P + kk];
            for (int i = kk + lane; i < n; i += 32) S[kk * P + i] = fma(-S[j * P + i], lkj, S[kk * P + i]);
        }
        __syncwarp();
    }
    return inf;
}

// x (rows over lanes: x0 row lane, x1 row lane + 32) <- L^{-1} x, then
// (both) L^{-T} x, with L in shared memory.
__device__ __forceinline__ void chol_solve_f64_warp(const double *S, int P, int n, int lane, double &x0, double &x1,
                                                    bool both) {
    for (int i = 0; i < n; ++i) {
        const double v = __shfl_sync(GLASS_FULL_MASK, i < 32 ? x0 : x1, i & 31);
        const double xi = v / S[i * P + i];
        if (lane == i) x0 = xi;
        else if (lane > i && lane < n) x0 = fma(-S[i * P + lane], xi, x0);
        if (lane + 32 == i) x1 = xi;
        else if (lane + 32 > i && lane + 32 < n) x1 = fma(-S[i * P + lane + 32], xi, x1);
    }
    if (!both) return;
    for (int i = n - 1; i >= 0; --i) {
        const double v = __shfl_sync(GLASS_FULL_MASK, i < 32 ? x0 : x1, i & 31);
        const double xi = v / S[i * P + i];
        if (lane == i) x0 = xi;
        else if (lane < i) x0 = fma(-S[lane * P + i], xi, x0);
        if (lane + 32 == i) x1 = xi;
        else if (lane + 32 < i) x1 = fma(-S[(lane + 32) * P + i], xi, x1);
    }
}

// COLS: many right-hand sides, one column per lane (x in a per-warp shared
// buffer of 32 columns), L read as broadcasts -- no shuffles or barriers in
// the sweeps; otherwise rows over lanes, one right-hand side at a time.
template <int OP, bool COLS>
__global__ void __launch_bounds__(256) k_chol_f64_warp(int n, int nrhs, double *A, int lda, long long sA, double *B,
                                                       int ldb, long long sB, int *info, int batch) {
    extern __shared__ double dsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, P = n | 1;
    double *S = dsm + w * (n + (COLS ? 32 : 0)) * P;
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= batch) return;
    double *a = A + b * sA;
    stage_f64(S, P, a, lda, n, lane, true);
    if (OP == 0 || OP == 2) {
        const int inf = potrf_f64_warp(S, P, n, lane);
        if (lane == 0) info[b] = inf;
        for (int e = lane; e < n * n; e += 32) {
            const int j = e / n, i = e - j * n;
            if (i >= j) a[(long long)j * lda + i] = S[j * P + i];
        }
    }
    if (OP == 0) return;
    double *bb = B + b * sB;
    if (COLS) {
        __syncwarp();
        double *X = S + n * P + lane * P;  // this lane's column
        for (int c = lane; c - lane < nrhs; c += 32) {
            const bool act = c < nrhs;
            if (act)
                for (int i = 0; i < n; ++i) X[i] = bb[(long long)c * ldb + i];
            for (int i = 0; i < n; ++i) {
                double s = X[i];
                for (int kk = 0; kk < i; ++kk) s = fma(-S[kk * P + i], X[kk], s);
                X[i] = s / S[i * P + i];
            }
            if (OP != 3)
                for (int i = n - 1; i >= 0; --i) {
                    double s = X[i];
                    for (int kk = i + 1; kk < n; ++kk) s = fma(-S[i * P + kk], X[kk], s);
                    X[i] = s / S[i * P + i];
                }
            if (act)
                for (int i = 0; i < n; ++i) bb[(long long)c * ldb + i] = X[i];
        }
        return;
    }
    for (int c = 0; c < nrhs; ++c) {
        double x0 = lane < n ? bb[(long long)c * ldb + lane] : 0.0;
        double x1 = lane + 32 < n ? bb[(long long)c * ldb + lane + 32] : 0.0;
        chol_solve_f64_warp(S, P, n, lane, x0, x1, OP != 3);
        if (lane < n) bb[(long long)c * ldb + lane] = x0;
        if (lane + 32 < n) bb[(long long)c * ldb + lane + 32] = x1;
    }
}

__global__ void __launch_bounds__(256) k_lu_f64_warp(int n, int nrhs, double *A, int lda, long long sA, int *ipiv,
                                                     double *B, int ldb, long long sB, int *info, int batch) {
    extern __shared__ double dsm[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, P = n | 1;
    double *S = dsm + w * n * P;
    int *pv_s = reinterpret_cast<int *>(dsm + (blockDim.x >> 5) * n * P) + w * 64;
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= batch) return;
    double *a = A + b * sA;
    stage_f64(S, P, a, lda, n, lane, false);
    int inf = 0;
    for (int j = 0; j < n; ++j) {
        // pivot: largest |a_ij| (i >= j), smallest i on ties, by a butterfly
        double v = -1.0;
        int vi = 0x7fffffff;
        for (int i = j + lane; i < n; i += 32) {
            const double t = fabs(S[j * P + i]);
            if (t > v) { v = t; vi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(GLASS_FULL_MASK, v, o);
            const int oi = __shfl_xor_sync(GLASS_FULL_MASK, vi, o);
            if (ov > v || (ov == v && oi < vi)) { v = ov; vi = oi; }
        }
        const int p = vi < n ? vi : j;  // no comparable candidate (NaN column): keep the row
        if (lane == 0) pv_s[j] = p;
        if (p != j)
            for (int c = lane; c < n; c += 32) {
                const double t = S[c * P + j];
                S[c * P + j] = S[c * P + p];
                S[c * P + p] = t;
            }
        __syncwarp();
        const double pv = S[j * P + j];
        if (pv == 0.0) {
            if (inf == 0) inf = j + 1;
        } else {
            for (int i = j + 1 + lane; i < n; i += 32) S[j * P + i] = S[j * P + i] / pv;
            __syncwarp();
            for (int c = j + 1; c < n; ++c) {
                const double ajc = S[c * P + j];
                for (int i = j + 1 + lane; i < n; i += 32) S[c * P + i] = fma(-S[j * P + i], ajc, S[c * P + i]);
            }
        }
        __syncwarp();
    }
    if (lane == 0) info[b] = inf;
    for (int j = lane; j < n; j += 32) ipiv[b * n + j] = pv_s[j];
    double *bb = B + b * sB;
    for (int c = 0; c < nrhs; ++c) {
        double x0 = lane < n ? bb[(long long)c * ldb + lane] : 0.0;
        double x1 = lane + 32 < n ? bb[(long long)c * ldb + lane + 32] : 0.0;
        for (int j = 0; j < n; ++j) {  // the interchanges in order
            const int p = pv_s[j];
            if (p != j) {
                const double xj = __shfl_sync(GLASS_FULL_MASK, j < 32 ? x0 : x1, j & 31);
                const double xp = __shfl_sync(GLASS_FULL_MASK, p < 32 ? x0 : x1, p & 31);
                if (lane == j) x0 = xp;
                if (lane == p) x0 = xj;
                if (lane + 32 == j) x1 = xp;
                if (lane + 32 == p) x1 = xj;
            }
        }
        for (int i = 0; i < n; ++i) {  // unit lower
            const double xi = __shfl_sync(GLASS_FULL_MASK, i < 32 ? x0 : x1, i & 31);
            if (lane > i && lane < n) x0 = fma(-S[i * P + lane], xi, x0);
            if (lane + 32 > i && lane + 32 < n) x1 = fma(-S[i * P + lane + 32], xi, x1);
        }
        for (int i = n - 1; i >= 0; --i) {  // upper, column-oriented
            const double xi = __shfl_sync(GLASS_FULL_MASK, i < 32 ? x0 : x1, i & 31) / S[i * P + i];
            if (lane == i) x0 = xi;
            else if (lane < i) x0 = fma(-S[i * P + lane], xi, x0);
            if (lane + 32 == i) x1 = xi;
            else if (lane + 32 < i) x1 = fma(-S[i * P + lane + 32], xi, x1);
        }
        if (lane < n) bb[(long long)c * ldb + lane] = x0;
        if (lane + 32 < n) bb[(long long)c * ldb + lane + 32] = x1;
    }
    for (int e = lane; e < n * n; e += 32) {
        const int j = e / n, i = e - j * n;
        a[(long long)j * lda + i] = S[j * P + i];
    }
}

constexpr size_t kMaxSmem = 227 * 1024;

size_t f64_warp_smem(int n, int pack, bool lu) {
    return (size_t)pack * (size_t)n * (n | 1) * 8 + (lu ? (size_t)pack * 64 * 4 : 0);
}

}  // namespace

bool feasible_f64(int op, int n, Placement pl) {
    if (n < 1 || n > 64) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (pl.scope == SCOPE_THREAD) return n <= kF64MaxThreadN;
    if (pl.scope != SCOPE_WARP) return false;
    if (op == GLASS_OP_GEMM) return true;
    return f64_warp_smem(n, pl.pack, op == GLASS_OP_GETRF_GETRS) <= kMaxSmem;
}

cudaError_t launch_gemm_f64(int m, int n, int k, const double *A, int lda, long long sA, const double *B, int ldb,
                            long long sB, double *C, int ldc, long long sC, int batch, Placement pl, cudaStream_t st) {
    const int mx = m > n ? (m > k ? m : k) : (n > k ? n : k);
    if (!feasible_f64(GLASS_OP_GEMM, mx, pl)) return cudaErrorInvalidConfiguration;
    if (pl.scope == SCOPE_THREAD) {
        const int th = 32 * pl.pack, grid = ceil_div(batch, th);
        if (mx <= 4) k_gemm_f64_thread<4><<<grid, th, 0, st>>>(m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch);
        else k_gemm_f64_thread<8><<<grid, th, 0, st>>>(m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch);
    } else {
        k_gemm_f64_warp<<<ceil_div(batch, pl.pack), 32 * pl.pack, 0, st>>>(m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC,
                                                                            batch);
    }
    return cudaPeekAtLastError();
}

// op: GLASS_OP_POTRF / POTRS / POSV / TRSM
cudaError_t launch_chol_f64(int op, int n, int nrhs, double *A, int lda, long long sA, double *B, int ldb, long long sB,
                            int *info, int batch, Placement pl, cudaStream_t st) {
    if (!feasible_f64(op, n, pl)) return cudaErrorInvalidConfiguration;
    const int kop = op == GLASS_OP_POTRF ? 0 : op == GLASS_OP_POTRS ? 1 : op == GLASS_OP_POSV ? 2 : 3;
    if (pl.scope == SCOPE_THREAD) {
        const int th = 32 * pl.pack, grid = ceil_div(batch, th);
#define GL_C(K, N) k_chol_f64_thread<K, N><<<grid, th, 0, st>>>(n, nrhs, A, lda, sA, B, ldb, sB, info, batch)
#define GL_CN(K) do { if (n <= 2) GL_C(K, 2); else if (n <= 4) GL_C(K, 4); else GL_C(K, 8); } while (0)
        switch (kop) {
            case 0: GL_CN(0); break;
            case 1: GL_CN(1); break;
            case 2: GL_CN(2); break;
            default: GL_CN(3); break;
        }
#undef GL_CN
#undef GL_C
        return cudaPeekAtLastError();
    }
    // many right-hand sides: a column per lane when the 32-column buffer fits
    const size_t smc = (size_t)pl.pack * (n + 32) * (n | 1) * 8;
    const bool cols = kop != 0 && nrhs >= 4 && smc <= kMaxSmem;
    const size_t sm = cols ? smc : f64_warp_smem(n, pl.pack, false);
    const int grid = ceil_div(batch, pl.pack), th = 32 * pl.pack;
#define GL_W(K, C)                                                                                         \
    do {                                                                                                   \
        cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(k_chol_f64_warp<K, C>), sm);          \
        if (e != cudaSuccess) return e;                                                                    \
        k_chol_f64_warp<K, C><<<grid, th, sm, st>>>(n, nrhs, A, lda, sA, B, ldb, sB, info, batch);         \
    } while (0)
    switch (kop) {
        case 0: GL_W(0, false); break;
        case 1: if (cols) GL_W(1, true); else GL_W(1, false); break;
        case 2: if (cols) GL_W(2, true); else GL_W(2, false); break;
        default: if (cols) GL_W(3, true); else GL_W(3, false); break;
    }
#undef GL_W
    return cudaPeekAtLastError();
}

cudaError_t launch_lu_f64(int n, int nrhs, double *A, int lda, long long sA, int *ipiv, double *B, int ldb, long long sB,
                          int *info, int batch, Placement pl, cudaStream_t st) {
    if (!feasible_f64(GLASS_OP_GETRF_GETRS, n, pl)) return cudaErrorInvalidConfiguration;
    if (pl.scope == SCOPE_THREAD) {
        const int th = 32 * pl.pack, grid = ceil_div(batch, th);
        if (n <= 2) k_lu_f64_thread<2><<<grid, th, 0, st>>>(n, nrhs, A, lda, sA, ipiv, B, ldb, sB, info, batch);
        else if (n <= 4) k_lu_f64_thread<4><<<grid, th, 0, st>>>(n, nrhs, A, lda, sA, ipiv, B, ldb, sB, info, batch);
        else k_lu_f64_thread<8><<<grid, th, 0, st>>>(n, nrhs, A, lda, sA, ipiv, B, ldb, sB, info, batch);
        return cudaPeekAtLastError();
    }
    const size_t sm = f64_warp_smem(n, pl.pack, true);
    cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(k_lu_f64_warp), sm);
    if (e != cudaSuccess) return e;
    k_lu_f64_warp<<<ceil_div(batch, pl.pack), 32 * pl.pack, sm, st>>>(n, nrhs, A, lda, sA, ipiv, B, ldb, sB, info,
                                                                       batch);
    return cudaPeekAtLastError();
}

}  // namespace glass
