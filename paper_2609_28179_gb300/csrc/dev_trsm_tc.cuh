// dev_trsm_tc.cuh -- blocked triangular solves with many right-hand sides
// and tensor-core updates, for orders 33..64: X = L^{-1} B (trsm) and
// X = L^{-T} L^{-1} B (potrs against a Cholesky factor).
//
// A team of T threads owns one problem: L (lower triangle, pitch LD) and
// 1/l_ii in shared memory, shared by the team; each warp solves chunks of 32
// right-hand sides held in its own shared-memory buffer (pitch LDB).  Per
// 16-row block p of the forward sweep:
//   1. X_p = L_pp^{-1} B_p on the SIMT pipe, one right-hand side per lane,
//      the 16 values in registers and L_pp read as 16-byte broadcasts;
//   2. B_q -= L_qp X_p for every later block q on the tensor cores
//      (mma.sync m16n8k8, 3xTF32 split, FP32 accumulation; four independent
//      16x8 accumulators per block).
// The backward sweep with L^T runs the same two steps from the last block
// up, with the diagonal solve in dot-product form and the updates reading
// L_qp^T.  Rows n..63 of L and of every buffer are zero and 1/l_ii is zero
// there, so the padded block stays zero.
#pragma once

#include "dev_chol_tc.cuh"

namespace glass {
namespace tctrsm {

using tcwarp::mma_tf32;
using tcwarp::split;

constexpr int NMAX = 64;
constexpr int LD = NMAX + 8;   // L: 8 mod 32, conflict-free A fragments
constexpr int LDB = NMAX + 4;  // B chunks: 4 mod 32, conflict-free C/B fragments and column loads
constexpr int CW = 32;  // right-hand sides per warp chunk

// Shared-memory floats of one problem for a team of T threads.
template <int T>
constexpr int floats() {
    return NMAX * LD + NMAX + (T / 32) * CW * LDB;
}

// Copy rows 0..n-1 of the first `cols` of `ncols` columns of a column-major
// operand (leading dimension ld) into dst (pitch P) with cp.async; zero
// the rest of the ncols x NMAX block.  `vec`: 16-byte copies (n, ld multiples
// of 4 and a 16-byte aligned base).  LOWER: skip the 16-byte groups that lie
// wholly above the diagonal (they are never read).  The caller waits.
template <bool LOWER>
__device__ __forceinline__ void stage_cols(float *dst, int P, const float *src, long long ld, int n, int cols,
                                           int ncols, bool vec, int rank, int T) {
    if (vec) {
        for (int e = rank; e < ncols * (NMAX / 4); e += T) {
            const int j = e >> 4, r = 4 * (e & 15);
            float *d = dst + j * P + r;
            if (j < cols && r < n) {
                if (!LOWER || r + 3 >= j) cp_async16(d, src + (long long)j * ld + r);
            } else {
                *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    } else {
        for (int e = rank; e < ncols * NMAX; e += T) {
            const int j = e >> 6, i = e & 63;
            float *d = dst + j * P + i;
            if (j < cols && i < n) {
                if (!LOWER || i >= j) cp_async4(d, src + (long long)j * ld + i);
            } else {
                *d = 0.f;
            }
        }
    }
}

// Copy the first `cols` columns (rows 0..n-1) of a chunk back to global.
__device__ __forceinline__ void store_cols(float *dst, long long ld, const float *src, int n, int cols, bool vec) {
    const int lane = threadIdx.x & 31;
    if (vec) {
        for (int e = lane; e < cols * (NMAX / 4); e += 32) {
            const int j = e >> 4, r = 4 * (e & 15);
            if (r < n) __stcs(reinterpret_cast<float4 *>(dst + (long long)j * ld + r),
                              *reinterpret_cast<const float4 *>(src + j * LDB + r));
        }
    } else {
        for (int e = lane; e < cols * NMAX; e += 32) {
            const int j = e >> 6, i = e & 63;
            if (i < n) dst[(long long)j * ld + i] = src[j * LDB + i];
        }
    }
}

__device__ __forceinline__ void load16(const float *p, float (&v)[16]) {
    const float4 *s = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float4 q = s[r];
        v[4 * r] = q.x;
        v[4 * r + 1] = q.y;
        v[4 * r + 2] = q.z;
        v[4 * r + 3] = q.w;
    }
}

__device__ __forceinline__ void store16(float *p, const float (&v)[16]) {
    float4 *d = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int r = 0; r < 4; ++r) d[r] = make_float4(v[4 * r], v[4 * r + 1], v[4 * r + 2], v[4 * r + 3]);
}

// Bs[rows 16q..16q+15] -= A X_p over the warp's 32 columns, where the 16x16
// operand A is L_qp (TRANS false) or L_pq^T (TRANS true).
template <bool TRANS>
__device__ __forceinline__ void update(const float *Ls, float *Bs, int p, int q) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    unsigned ah[2][4], al[2][4];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int k0 = 16 * p + 8 * kk + t;
        float a[4];
        if (!TRANS) {  // A(m, k) = L[16q + m][16p + k]
            a[0] = Ls[k0 * LD + 16 * q + g];
            a[1] = Ls[k0 * LD + 16 * q + g + 8];
            a[2] = Ls[(k0 + 4) * LD + 16 * q + g];
            a[3] = Ls[(k0 + 4) * LD + 16 * q + g + 8];
        } else {  // A(m, k) = L[16p + k][16q + m]
            a[0] = Ls[(16 * q + g) * LD + k0];
            a[1] = Ls[(16 * q + g + 8) * LD + k0];
            a[2] = Ls[(16 * q + g) * LD + k0 + 4];
            a[3] = Ls[(16 * q + g + 8) * LD + k0 + 4];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) split(-a[r], ah[kk][r], al[kk][r]);
    }
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const float *c = Bs + (8 * nt + 2 * t) * LDB + 16 * q + g;
        acc[nt][0] = c[0];
        acc[nt][1] = c[LDB];
        acc[nt][2] = c[8];
        acc[nt][3] = c[LDB + 8];
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        unsigned bh[4][2], bl[4][2];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const float *x = Bs + (8 * nt + g) * LDB + 16 * p + 8 * kk + t;
            split(x[0], bh[nt][0], bl[nt][0]);
            split(x[4], bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_tf32(acc[nt], al[kk], bh[nt]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_tf32(acc[nt], ah[kk], bl[nt]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_tf32(acc[nt], ah[kk], bh[nt]);
    }
    float *wb = opaque(Bs);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        float *c = wb + (8 * nt + 2 * t) * LDB + 16 * q + g;
        c[0] = acc[nt][0];
        c[LDB] = acc[nt][1];
        c[8] = acc[nt][2];
        c[LDB + 8] = acc[nt][3];
    }
}

// Bs <- L^{-1} Bs (the warp's 32 columns).
__device__ __forceinline__ void forward(const float *Ls, const float *dv, float *Bs, int n) {
    const int lane = threadIdx.x & 31;
    const int nb = (n + 15) >> 4;
    for (int p = 0; p < nb; ++p) {
        float x[16];
        load16(Bs + lane * LDB + 16 * p, x);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float l[16];
            load16(Ls + (16 * p + r) * LD + 16 * p, l);
            x[r] *= dv[16 * p + r];
#pragma unroll
            for (int s = 0; s < 16; ++s)
                if (s > r) x[s] = fmaf(-l[s], x[r], x[s]);
        }
        store16(opaque(Bs) + lane * LDB + 16 * p, x);
        __syncwarp();
        for (int q = p + 1; q < nb; ++q) update<false>(Ls, Bs, p, q);
        __syncwarp();
    }
}

// Bs <- L^{-T} Bs (the warp's 32 columns).
__device__ __forceinline__ void backward_t(const float *Ls, const float *dv, float *Bs, int n) {
    const int lane = threadIdx.x & 31;
    const int nb = (n + 15) >> 4;
    for (int p = nb - 1; p >= 0; --p) {
        float x[16];
        load16(Bs + lane * LDB + 16 * p, x);
#pragma unroll
        for (int r = 15; r >= 0; --r) {
            float l[16];
            load16(Ls + (16 * p + r) * LD + 16 * p, l);
            float s = x[r];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k > r) s = fmaf(-l[k], x[k], s);
            x[r] = s * dv[16 * p + r];
        }
        store16(opaque(Bs) + lane * LDB + 16 * p, x);
        __syncwarp();
        for (int q = 0; q < p; ++q) update<true>(Ls, Bs, p, q);
        __syncwarp();
    }
}

}  // namespace tctrsm
}  // namespace glass
