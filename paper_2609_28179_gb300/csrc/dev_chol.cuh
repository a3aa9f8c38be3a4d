// dev_chol.cuh -- composable device primitives for the Cholesky family
// (potrf, potrs, trsm; posv = potrf + potrs) at the three execution scopes
// of Sec. III-A:
//   glass::thread : one problem per thread, operand in registers (n <= 16);
//   glass::warp   : one problem per warp, row i of the operand in the
//                   registers of lane i % 32 (two rows per lane above 32),
//                   columns broadcast through a per-warp shared buffer
//                   (shuffles at two rows per lane);
//                   many right-hand sides: one column of X per thread with
//                   L broadcast from shared memory;
//   block scope   : a 64-thread row team per problem (dev_rows.cuh).
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
// The trailing update at step j needs l_kj from the lane that holds row k.
// Up to NMAX = 32 that column goes through the warp's NMAX-float shared
// buffer `col` (16-byte aligned): every lane publishes its l_ij and reads
// the l_kj back as 16-byte broadcasts (one load per four columns instead of
// one shuffle per column).  At NMAX = 64 (two rows per lane) the shuffle
// form keeps the 128-entry row block in registers, so it is used there.
// Returns info, identical in every lane.
template <int NMAX>
__device__ __forceinline__ int potrf(float (&a)[Rows<NMAX>::R][NMAX], float (&rd)[Rows<NMAX>::R], int n,
                                     bool fp64diag, float *col) {
    constexpr int R = Rows<NMAX>::R;
    constexpr bool kSmem = NMAX <= 32;
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
                if (kSmem && i < NMAX) col[i] = a[q][j];
            }
            if constexpr (kSmem) {
                __syncwarp();
#pragma unroll
                for (int k4 = (j + 1) / 4; k4 < NMAX / 4; ++k4) {
                    const float4 v = *reinterpret_cast<const float4 *>(col + 4 * k4);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = 4 * k4 + u;
                        if (k > j) {
                            const int i = lane;
                            if (i >= k) a[0][k] = fmaf(-a[0][j], vv[u], a[0][k]);
                        }
                    }
                }
                __syncwarp();
            } else {
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

// Triangular solves with many right-hand sides: each thread owns one
// column x[0..NMAX) of X and reads L (column-major, leading dimension
// NMAX, 16-byte aligned, shared memory) and dinv (shared) by broadcast.
// x <- L^{-1} x, right-looking: after x_i is final, the trailing entries
// take -l_ri x_i, the l_ri read four at a time from column i.
template <int NMAX>
__device__ __forceinline__ void forward_cols(const float *Ls, const float *dinv_s, float (&x)[NMAX], int n) {
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
            x[i] *= dinv_s[i];
            const float4 *c4 = reinterpret_cast<const float4 *>(Ls + i * NMAX);
#pragma unroll
            for (int q4 = (i + 1) / 4; q4 < NMAX / 4; ++q4) {
                const float4 v = c4[q4];
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = 4 * q4 + u;
                    if (r > i && r < n) x[r] = fmaf(-vv[u], x[i], x[r]);
                }
            }
        }
    }
}

// x <- L^{-T} x, dot-product form: x_i = (y_i - sum_{k>i} l_ki x_k) / l_ii,
// column i of L read four at a time, two partial sums for ILP.
template <int NMAX>
__device__ __forceinline__ void backward_t_cols(const float *Ls, const float *dinv_s, float (&x)[NMAX], int n) {
#pragma unroll
    for (int i = NMAX - 1; i >= 0; --i) {
        if (i < n) {
            const float4 *c4 = reinterpret_cast<const float4 *>(Ls + i * NMAX);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int q4 = (i + 1) / 4; q4 < NMAX / 4; ++q4) {
                const float4 v = c4[q4];
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = 4 * q4 + u;
                    if (k > i && k < n) {
                        if (u & 1) s1 = fmaf(vv[u], x[k], s1);
                        else s0 = fmaf(vv[u], x[k], s0);
                    }
                }
            }
            x[i] = (x[i] - (s0 + s1)) * dinv_s[i];
        }
    }
}

}  // namespace warp

}  // namespace glass
