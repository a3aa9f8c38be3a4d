// dev_lu.cuh -- LU factorization with partial pivoting and the matching
// solve, at thread, warp and block scope (Sec. III-A scopes; Sec. III-B
// "factorizations, and linear solves").
//
// Pivot rule (all scopes): at step j the row with the largest |a_ij| among
// the rows still to be eliminated wins, the smallest current row index on
// ties; ipiv[j] records the exchanged row in sequential-swap form.
//
// Warp scope (orders up to 16, two problems per warp) keeps every row in the
// registers of one lane and never moves it: a pivot exchange only relabels
// logical positions (pos), the
// multipliers stay with their physical row, and the final packed factor is
// written out row by row at each row's logical position.  This is the same
// factorization as the explicit-swap algorithm (rows carry their
// multipliers with them in both), without 2n shuffles per exchange.
#pragma once

#include "common.cuh"

namespace glass {
namespace thread {

// Full n x n matrix a[i][k] in registers.  piv[j] = row exchanged at step j,
// rinv[j] = 1 / u_jj.  Returns info (first exactly-zero pivot).
template <int NMAX, bool EXACT>
__device__ __forceinline__ int getrf(float (&a)[NMAX][NMAX], int (&piv)[NMAX], float (&rinv)[NMAX], int n_rt) {
    const int n = EXACT ? NMAX : n_rt;
    int info = 0;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            int p = j;
            float best = fabsf(a[j][j]);
#pragma unroll
            for (int r = j + 1; r < NMAX; ++r)
                if (r < n) {
                    const float v = fabsf(a[r][j]);
                    if (v > best) { best = v; p = r; }
                }
            piv[j] = p;
            // exchange rows j and p (p >= j, a runtime index: select chains)
#pragma unroll
            for (int c = 0; c < NMAX; ++c) {
                const float vj = a[j][c];
                float vp = vj;
#pragma unroll
                for (int r = j + 1; r < NMAX; ++r)
                    if (r == p) vp = a[r][c];
#pragma unroll
                for (int r = j + 1; r < NMAX; ++r)
                    if (r == p) a[r][c] = vj;
                a[j][c] = vp;
            }
            const float pv = a[j][j];
            if (pv == 0.f) {
                if (info == 0) info = j + 1;
                rinv[j] = 0.f;
            } else {
                const float rc = 1.0f / pv;
                rinv[j] = rc;
#pragma unroll
                for (int r = j + 1; r < NMAX; ++r) {
                    if (r < n) {
                        a[r][j] *= rc;
#pragma unroll
                        for (int c = j + 1; c < NMAX; ++c)
                            if (c < n) a[r][c] = fmaf(-a[r][j], a[j][c], a[r][c]);
                    }
                }
            }
        }
    }
    return info;
}

// x <- U^{-1} L^{-1} P x for one right-hand side.
template <int NMAX, bool EXACT>
__device__ __forceinline__ void getrs(const float (&a)[NMAX][NMAX], const int (&piv)[NMAX], const float (&rinv)[NMAX],
                                      float (&x)[NMAX], int n_rt) {
    const int n = EXACT ? NMAX : n_rt;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            const int p = piv[j];
            float vp = x[j];
#pragma unroll
            for (int r = j + 1; r < NMAX; ++r)
                if (r == p) vp = x[r];
#pragma unroll
            for (int r = j + 1; r < NMAX; ++r)
                if (r == p) x[r] = x[j];
            x[j] = vp;
        }
    }
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
        if (i < n)
#pragma unroll
            for (int r = i + 1; r < NMAX; ++r)
                if (r < n) x[r] = fmaf(-a[r][i], x[i], x[r]);
#pragma unroll
    for (int i = NMAX - 1; i >= 0; --i)
        if (i < n) {
            x[i] *= rinv[i];
#pragma unroll
            for (int r = 0; r < i; ++r) x[r] = fmaf(-a[r][i], x[i], x[r]);
        }
}

}  // namespace thread

// ------------------------------------------------------------ half-warp
// Orders <= 16 with two problems per warp: lanes 16 h .. 16 h + 15 hold the
// rows of problem h (row r in lane 16 h + r).  The pivot rule of every scope
// -- largest |a_ij| among the rows not yet eliminated, smallest logical
// position on ties -- with the reductions as butterflies inside each
// half (shuffle distances 8, 4, 2, 1 never cross halves).  A zero pivot takes
// the same path as any other (its multipliers are exactly zero: every
// candidate is zero), so the two halves never diverge.
namespace half {

__device__ __forceinline__ unsigned half_max(unsigned v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(GLASS_FULL_MASK, v, o));
    return v;
}
__device__ __forceinline__ unsigned half_min(unsigned v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(GLASS_FULL_MASK, v, o));
    return v;
}

// a[*]: row r = lane % 16 of this half's problem; pos receives the row's
// final logical position.  sm: this half's shared scratch, 2 * NMAX words
// (pp[j] = row chosen at step j, prc[j] = 1 / u_jj).  ipiv_out receives
// ipiv[0..n) (lane 0 of the half writes).  Returns info.
template <int NMAX>
__device__ __forceinline__ int getrf(float (&a)[NMAX], int &pos, int *sm, int *ipiv_out, int n) {
    static_assert(NMAX <= 16, "half-warp: orders up to 16");
    const int lane = threadIdx.x & 31, r = lane & 15, base = lane & 16;
    int *pp = sm;
    float *prc = reinterpret_cast<float *>(sm + NMAX);
    bool done = r >= n;
    pos = r;
    int info = 0;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            const unsigned key = done ? 0u : __float_as_uint(fabsf(a[j])) + 1u;
            const unsigned kmax = half_max(key);
            const int ppos = (int)half_min(key == kmax ? (unsigned)pos : 0xffffffffu);
            const unsigned m = __ballot_sync(GLASS_FULL_MASK, !done && pos == ppos);
            const int pphys = __ffs((m >> base) & 0xffffu) - 1;  // the winner's row in this half
            if (ipiv_out != nullptr && r == 0) ipiv_out[j] = ppos;
            if (pos == j) pos = ppos;
            if (r == pphys) { pos = j; done = true; }
            const float pv = __shfl_sync(GLASS_FULL_MASK, a[j], base + pphys);
            const float rc = pv != 0.f ? 1.0f / pv : 0.f;
            if (r == 0) { pp[j] = pphys; prc[j] = rc; }
            if (pv == 0.f && info == 0) info = j + 1;
            const float mj = done ? 0.f : a[j] * rc;
            if (!done) a[j] = mj;
#pragma unroll
            for (int k = 0; k < NMAX; ++k) {  // fixed range: keeps a[] in registers
                if (k > j && k < n) {
                    const float pk = __shfl_sync(GLASS_FULL_MASK, a[k], base + pphys);
                    a[k] = fmaf(-mj, pk, a[k]);
                }
            }
        }
    }
    __syncwarp();
    return info;
}

// One right-hand side held by physical row (x = b of row lane % 16, the
// row's original index): on return x is the solution component at logical
// position pos.
template <int NMAX>
__device__ __forceinline__ void getrs(const float (&a)[NMAX], int pos, const int *sm, float &x, int n) {
    const int lane = threadIdx.x & 31, r = lane & 15, base = lane & 16;
    const int *pp = sm;
    const float *prc = reinterpret_cast<const float *>(sm + NMAX);
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            const float yj = __shfl_sync(GLASS_FULL_MASK, x, base + pp[j]);
            if (pos > j && r < n) x = fmaf(-a[j], yj, x);
        }
    }
#pragma unroll
    for (int j = NMAX - 1; j >= 0; --j) {
        if (j < n) {
            const int pj = pp[j];
            const float xj = __shfl_sync(GLASS_FULL_MASK, x, base + pj) * prc[j];
            if (r == pj) x = xj;
            else if (pos < j && r < n) x = fmaf(-a[j], xj, x);
        }
    }
}

}  // namespace half

}  // namespace glass
