// dev_chol.cuh -- composable device primitives for the Cholesky family
// (potrf, potrs, trsm; posv = potrf + potrs) at the three execution scopes
// of Sec. III-A:
//   glass::thread : one problem per thread, operand in registers (n <= 16);
//   glass::warp   : one problem per warp, row i of the operand in the
//                   registers of lane i % 32 (two rows per lane above 32),
//                   columns broadcast with shuffles;
//   glass::block  : one problem per team of T threads, operand resident in
//                   shared memory, steps separated by named barriers.
// All scopes follow one convention: lower factor, column-major operand,
// L L^T = A (the paper's shared-convention rule, Sec. III-A).  The
// arithmetic is the right-looking form of the textbook recurrences
// (Sec. III-B factorizations and triangular solves); the diagonal is
// inverted once and applied by multiplication.
#pragma once

#include "common.cuh"

namespace glass {

// Packed lower triangle, column-major: (i, j), i >= j, at idx(i, j).
template <int N>
struct Tri {
    static constexpr int size = N * (N + 1) / 2;
    __host__ __device__ static constexpr int idx(int i, int j) {
        return j * N - j * (j - 1) / 2 + (i - j);
    }
};

namespace thread {

// In-place Cholesky of the packed lower triangle a (order n <= NMAX; with
// EXACT the order is NMAX).  dinv[j] receives 1 / l_jj.  Returns info.
template <int NMAX, bool EXACT>
__device__ __forceinline__ int potrf(float (&a)[Tri<NMAX>::size], float (&dinv)[NMAX], int n_rt,
                                     bool fp64diag) {
    using T = Tri<NMAX>;
    const int n = EXACT ? NMAX : n_rt;
    int info = 0;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            const float d = a[T::idx(j, j)];
            if (!(d > 0.f) && info == 0) info = j + 1;
            float l, r;
            chol_diag(d, fp64diag, l, r);
            a[T::idx(j, j)] = l;
            dinv[j] = r;
#pragma unroll
            for (int i = j + 1; i < NMAX; ++i)
                if (i < n) a[T::idx(i, j)] *= r;
#pragma unroll
            for (int k = j + 1; k < NMAX; ++k)
#pragma unroll
                for (int i = k; i < NMAX; ++i)
                    if (i < n) a[T::idx(i, k)] = fmaf(-a[T::idx(i, j)], a[T::idx(k, j)], a[T::idx(i, k)]);
        }
    }
    return info;
}

// x <- L^{-1} x (forward substitution, non-unit diagonal via dinv).
template <int NMAX, bool EXACT>
__device__ __forceinline__ void forward(const float (&a)[Tri<NMAX>::size], const float (&dinv)[NMAX],
                                        float (&x)[NMAX], int n_rt) {
    using T = Tri<NMAX>;
    const int n = EXACT ? NMAX : n_rt;
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
            x[i] *= dinv[i];
#pragma unroll
            for (int r = i + 1; r < NMAX; ++r)
                if (r < n) x[r] = fmaf(-a[T::idx(r, i)], x[i], x[r]);
        }
    }
}

// x <- L^{-T} x (backward substitution with the transposed factor).
template <int NMAX, bool EXACT>
__device__ __forceinline__ void backward_t(const float (&a)[Tri<NMAX>::size], const float (&dinv)[NMAX],
                                           float (&x)[NMAX], int n_rt) {
    using T = Tri<NMAX>;
    const int n = EXACT ? NMAX : n_rt;
#pragma unroll
    for (int i = NMAX - 1; i >= 0; --i) {
        if (i < n) {
            x[i] *= dinv[i];
#pragma unroll
            for (int r = 0; r < i; ++r) x[r] = fmaf(-a[T::idx(i, r)], x[i], x[r]);
        }
    }
}

}  // namespace thread

namespace warp {

template <int NMAX>
struct Rows {
    static constexpr int R = (NMAX + 31) / 32;  // rows held per lane
};

// In-place Cholesky with row lane+32r of the operand in a[r][*] (only the
// entries k <= row are meaningful).  rd[r] receives 1 / l_rr of that row.
// Returns info, identical in every lane.
template <int NMAX>
__device__ __forceinline__ int potrf(float (&a)[Rows<NMAX>::R][NMAX], float (&rd)[Rows<NMAX>::R], int n,
                                     bool fp64diag) {
    constexpr int R = Rows<NMAX>::R;
    const int lane = threadIdx.x & 31;
    int info = 0;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            const float d = __shfl_sync(GLASS_FULL_MASK, a[j / 32][j], j % 32);
            if (!(d > 0.f) && info == 0) info = j + 1;
            float l, r;
            chol_diag(d, fp64diag, l, r);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (i == j) { a[q][j] = l; rd[q] = r; }
                else if (i > j) a[q][j] *= r;
            }
#pragma unroll
            for (int k = j + 1; k < NMAX; ++k) {
                if (k < n) {
                    const float lk = __shfl_sync(GLASS_FULL_MASK, a[k / 32][j], k % 32);
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int i = lane + 32 * q;
                        if (i >= k) a[q][k] = fmaf(-a[q][j], lk, a[q][k]);
                    }
                }
            }
        }
    }
    return info;
}

// One right-hand side distributed like the rows (x[r] is row lane+32r):
// x <- L^{-1} x.
template <int NMAX>
__device__ __forceinline__ void forward(const float (&a)[Rows<NMAX>::R][NMAX], const float (&rd)[Rows<NMAX>::R],
                                        float (&x)[Rows<NMAX>::R], int n) {
    constexpr int R = Rows<NMAX>::R;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
            const float yi = __shfl_sync(GLASS_FULL_MASK, x[i / 32] * rd[i / 32], i % 32);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = lane + 32 * q;
                if (row == i) x[q] = yi;
                else if (row > i) x[q] = fmaf(-a[q][i], yi, x[q]);
            }
        }
    }
}

// x <- L^{-T} x: x_i = (y_i - sum_{k>i} l_ki x_k) / l_ii, the sum reduced
// across the lanes that hold rows k > i.
template <int NMAX>
__device__ __forceinline__ void backward_t(const float (&a)[Rows<NMAX>::R][NMAX], const float (&rd)[Rows<NMAX>::R],
                                           float (&x)[Rows<NMAX>::R], int n) {
    constexpr int R = Rows<NMAX>::R;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = NMAX - 1; i >= 0; --i) {
        if (i < n) {
            float part = 0.f;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int row = lane + 32 * q;
                if (row > i && row < n) part = fmaf(a[q][i], x[q], part);
            }
            const float s = warp_sum(part);
            const float xi = __shfl_sync(GLASS_FULL_MASK, (x[i / 32] - s) * rd[i / 32], i % 32);
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (lane + 32 * q == i) x[q] = xi;
        }
    }
}

// Triangular solve with many right-hand sides: lane c owns column c of X
// (x[0..NMAX)) and reads L (column-major, leading dimension ldl, in shared
// memory) and dinv (shared) by broadcast.  x <- L^{-1} x.
template <int NMAX>
__device__ __forceinline__ void forward_cols(const float *Ls, int ldl, const float *dinv_s,
                                             float (&x)[NMAX], int n) {
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
            x[i] *= dinv_s[i];
            const float *col = Ls + i * ldl;
#pragma unroll
            for (int r = i + 1; r < NMAX; ++r)
                if (r < n) x[r] = fmaf(-col[r], x[i], x[r]);
        }
    }
}

}  // namespace warp

namespace block {

// Team of T threads on one problem resident in shared memory (column-major,
// leading dimension lda).  rank = thread index within the team; bar = the
// team's named barrier.  Every function ends with the team synchronised.

// Threads laid out as TI rows x TK column groups for trailing updates.
template <int T>
struct Grid2 {
    static constexpr int TI = T >= 64 ? 64 : T;
    static constexpr int TK = T / TI;
};

template <int T>
__device__ __forceinline__ int potrf(float *a, int lda, int n, int rank, int bar, bool fp64diag,
                                     float *dinv_s) {
    using G = Grid2<T>;
    int info = 0;
    const int ti = rank % G::TI, tk = rank / G::TI;
    for (int j = 0; j < n; ++j) {
        const float d = a[j * lda + j];
        if (!(d > 0.f) && info == 0) info = j + 1;
        float l, r;
        chol_diag(d, fp64diag, l, r);
        team_sync<T>(bar);  // everyone has read a_jj
        if (rank == 0) { a[j * lda + j] = l; dinv_s[j] = r; }
        for (int i = j + 1 + rank; i < n; i += T) a[j * lda + i] *= r;
        team_sync<T>(bar);
        for (int k = j + 1 + tk; k < n; k += G::TK) {
            const float lkj = a[j * lda + k];
            for (int i = ti; i < n; i += G::TI)
                if (i >= k) a[k * lda + i] = fmaf(-a[j * lda + i], lkj, a[k * lda + i]);
        }
        team_sync<T>(bar);
    }
    return info;
}

// dinv_s[i] = 1 / l_ii for a given factor.
template <int T>
__device__ __forceinline__ void diag_inverse(const float *a, int lda, int n, int rank, int bar,
                                             float *dinv_s) {
    for (int i = rank; i < n; i += T) dinv_s[i] = 1.0f / a[i * lda + i];
    team_sync<T>(bar);
}

// One right-hand side x (shared) <- L^{-1} x, rows updated in parallel.
template <int T>
__device__ __forceinline__ void forward(const float *a, int lda, const float *dinv_s, float *x, int n,
                                        int rank, int bar, bool unit = false) {
    for (int i = 0; i < n; ++i) {
        const float yi = unit ? x[i] : x[i] * dinv_s[i];
        for (int r = i + 1 + rank; r < n; r += T) x[r] = fmaf(-a[i * lda + r], yi, x[r]);
        team_sync<T>(bar);
        if (rank == 0) x[i] = yi;
    }
    team_sync<T>(bar);
}

// One right-hand side x (shared) <- L^{-T} x.
template <int T>
__device__ __forceinline__ void backward_t(const float *a, int lda, const float *dinv_s, float *x, int n,
                                           int rank, int bar) {
    for (int i = n - 1; i >= 0; --i) {
        const float xi = x[i] * dinv_s[i];
        for (int r = rank; r < i; r += T) x[r] = fmaf(-a[r * lda + i], xi, x[r]);
        team_sync<T>(bar);
        if (rank == 0) x[i] = xi;
    }
    team_sync<T>(bar);
}

}  // namespace block
}  // namespace glass
