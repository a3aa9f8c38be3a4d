// dev_chol_tc.cuh -- warp-scope blocked Cholesky with tensor-core trailing
// updates, for orders 33..64 (below that the register form is faster).
//
// One warp owns one problem held in its shared memory, column-major with
// pitch LD = NMAX + 8 (LD = 8 mod 32: every TF32 fragment load of the MMA
// touches 32 distinct banks).  The factorization runs over 16-column panels:
//   1. panel: the 16 columns c0..c0+15 (rows c0..n-1) are factored on the
//      SIMT pipe in registers (row i in lane i % 32), right-looking, with
//      the same diagonal rules as every other scope (Sec. III-B
//      factorizations; LAPACK info);
//   2. trailing update A22 -= L21 L21^T on the tensor cores: mma.sync
//      m16n8k8 TF32 over the 16x8 tiles of A22 that meet its lower
//      triangle, each product split 3xTF32 (a = a_hi + a_lo; hi*hi + hi*lo +
//      lo*hi) so the update keeps FP32-level accuracy; FP32 accumulation.
// Panel and tile loops run at run time, so the code stays small (the fully
// unrolled register form of the 64-column factorization spends a quarter of
// its stalls on instruction fetch).  Rows and columns from n to NMAX are
// zero, which keeps every padded tile update a no-op.
#pragma once

#include "common.cuh"

namespace glass {
namespace tcwarp {

__device__ __forceinline__ unsigned tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void split(float x, unsigned &hi, unsigned &lo) {
    hi = tf32(x);
    lo = tf32(x - __uint_as_float(hi));
}

template <int NMAX>
struct Shape {
    static constexpr int LD = NMAX + 8;
    static constexpr int R = NMAX / 32;  // rows per lane
};

// In-place Cholesky of the lower triangle of As (order n <= NMAX); dv[j]
// receives 1 / l_jj.  Returns info (uniform).
template <int NMAX>
__device__ __forceinline__ int potrf(float *As, int n, float *dv, bool fp64diag) {
    constexpr int LD = Shape<NMAX>::LD;
    constexpr int R = Shape<NMAX>::R;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    int info = 0;
    for (int c0 = 0; c0 < n; c0 += 16) {
        // ---- 1. panel on the SIMT pipe
        float p[R][16];
#pragma unroll
        for (int q = 0; q < R; ++q)
#pragma unroll
            for (int k = 0; k < 16; ++k) p[q][k] = As[(c0 + k) * LD + lane + 32 * q];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int cj = c0 + j;
            if (cj < n) {
                const int qj = cj >> 5;
                float dsel = p[0][j];
#pragma unroll
                for (int q = 1; q < R; ++q)
                    if (qj == q) dsel = p[q][j];
                const float d = __shfl_sync(GLASS_FULL_MASK, dsel, cj & 31);
                if (!(d > 0.f) && info == 0) info = cj + 1;
                float l, r;
                chol_diag(d, fp64diag, l, r);
                if (lane == 0) dv[cj] = r;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int i = lane + 32 * q;
                    if (i == cj) p[q][j] = l;
                    else if (i > cj) p[q][j] *= r;
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) {  // fixed range: keeps p[][] in registers
                    const int ck = c0 + k;
                    if (k > j && ck < n) {
                        const int qk = ck >> 5;
                        float sel = p[0][j];
#pragma unroll
                        for (int q = 1; q < R; ++q)
                            if (qk == q) sel = p[q][j];
                        const float lkj = __shfl_sync(GLASS_FULL_MASK, sel, ck & 31);
#pragma unroll
                        for (int q = 0; q < R; ++q)
                            if (lane + 32 * q >= ck) p[q][k] = fmaf(-p[q][j], lkj, p[q][k]);
                    }
                }
            }
        }
        float *wp = opaque(As);
#pragma unroll
        for (int q = 0; q < R; ++q)
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int i = lane + 32 * q;
                if (i >= c0 + k && i < n) wp[(c0 + k) * LD + i] = p[q][k];
            }
        __syncwarp();
        // ---- 2. trailing update on the tensor cores
        const int r0 = c0 + 16;
        for (int R0 = r0; R0 < n; R0 += 16) {
            unsigned ah[2][4], al[2][4];
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const float *col = As + (c0 + 8 * kk + t) * LD;
                split(-col[R0 + g], ah[kk][0], al[kk][0]);
                split(-col[R0 + g + 8], ah[kk][1], al[kk][1]);
                split(-col[4 * LD + R0 + g], ah[kk][2], al[kk][2]);
                split(-col[4 * LD + R0 + g + 8], ah[kk][3], al[kk][3]);
            }
            for (int C0 = r0; C0 < n && C0 <= R0 + 15; C0 += 8) {
                float *c = As + (C0 + 2 * t) * LD + R0 + g;
                float acc[4] = {c[0], c[LD], c[8], c[LD + 8]};
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const float *col = As + (c0 + 8 * kk + t) * LD;
                    unsigned bh[2], bl[2];
                    split(col[C0 + g], bh[0], bl[0]);
                    split(col[4 * LD + C0 + g], bh[1], bl[1]);
                    mma_tf32(acc, al[kk], bh);
                    mma_tf32(acc, ah[kk], bl);
                    mma_tf32(acc, ah[kk], bh);
                }
                c[0] = acc[0];
                c[LD] = acc[1];
                c[8] = acc[2];
                c[LD + 8] = acc[3];
            }
        }
        __syncwarp();
    }
    return info;
}

// One right-hand side held like the rows (x[q] = row lane + 32q) against L
// in shared memory: x <- L^{-1} x, then x <- L^{-T} x.
template <int NMAX>
__device__ __forceinline__ void potrs(const float *As, const float *dv, float (&x)[Shape<NMAX>::R], int n) {
    constexpr int LD = Shape<NMAX>::LD;
    constexpr int R = Shape<NMAX>::R;
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < n; ++i) {
        const int qi = i >> 5;
        float sel = x[0];
#pragma unroll
        for (int q = 1; q < R; ++q)
            if (qi == q) sel = x[q];
        const float yi = __shfl_sync(GLASS_FULL_MASK, sel, i & 31) * dv[i];
        const float *col = As + i * LD;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = lane + 32 * q;
            if (row == i) x[q] = yi;
            else if (row > i && row < n) x[q] = fmaf(-col[row], yi, x[q]);
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        const float *col = As + i * LD;
        float part = 0.f;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = lane + 32 * q;
            if (row > i && row < n) part = fmaf(col[row], x[q], part);
        }
        const float s = warp_sum(part);
        const int qi = i >> 5;
        float sel = x[0];
#pragma unroll
        for (int q = 1; q < R; ++q)
            if (qi == q) sel = x[q];
        const float xi = (__shfl_sync(GLASS_FULL_MASK, sel, i & 31) - s) * dv[i];
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (lane + 32 * q == i) x[q] = xi;
    }
}

}  // namespace tcwarp
}  // namespace glass
