// dev_lu_tc.cuh -- warp-scope blocked LU with partial pivoting and
// tensor-core trailing updates, for orders 17..64 (NMAX 32 or 64).
//
// One warp owns one problem in its shared memory (column-major, pitch
// LD = NMAX + 8, rows and columns beyond n zero).  Per 16-column panel:
//   1. the panel (rows c0..n-1) is factored in registers, row i in lane
//      i % 32; the pivot of column j is the largest |a_ij| among the rows not
//      yet eliminated, the smallest current row index on ties, and rows never
//      move inside the panel -- only their logical positions change (the same
//      rule and result as explicit interchanges);
//   2. the rows c0..n-1 of every other column, and the record of which
//      original row each logical row holds, are permuted to the panel's final
//      order, so logical and physical rows agree again (the interchanges
//      LAPACK applies to the columns left and right of a panel);
//   3. U12 = L11^{-1} A12 (unit lower, one column per lane);
//   4. A22 -= L21 U12 on the tensor cores: mma.sync m16n8k8, 3xTF32 split,
//      FP32 accumulation, two independent accumulator tiles per step.
// Once c0 >= 32 the rows held in the first register slot are all eliminated,
// so the panel and the interchanges run on the second slot only (QLO = 1).
// ipiv is produced in sequential-interchange form (Sec. III-B
// factorizations; the xGETF2 step order of the oracle), info on the first
// exactly zero pivot.
#pragma once

#include "dev_chol_tc.cuh"

namespace glass {
namespace tclu {

using tcwarp::mma_tf32;
using tcwarp::split;

// Pitch NMAX + 8 (8 mod 32): the L21 fragments load conflict free.  (NMAX + 4
// makes the accumulator tiles and the U12 solve conflict free instead and
// measured 5-8 % slower.)
template <int NMAX>
struct Shape {
    static constexpr int LD = NMAX + 8;
    static constexpr int R = NMAX / 32;
};

// Steps 1 and 2 for the panel at c0; rows held in slots q >= QLO.
template <int NMAX, int QLO>
__device__ __forceinline__ void panel(float *As, int *prow, int n, int c0, int *ipiv_s, float *dv, int &info) {
    constexpr int LD = Shape<NMAX>::LD;
    constexpr int R = Shape<NMAX>::R;
    const int lane = threadIdx.x & 31;
    float p[R][16];
    int pos[R];
    bool done[R];
#pragma unroll
    for (int q = QLO; q < R; ++q) {
        const int row = lane + 32 * q;
        pos[q] = row;
        done[q] = row < c0 || row >= n;
#pragma unroll
        for (int k = 0; k < 16; ++k) p[q][k] = As[(c0 + k) * LD + row];
    }
    // this lane's candidate for column j: largest |a|, then smallest position
    auto candidate = [&](int j, unsigned &key, unsigned &kpos, int &kq) {
        key = 0;
        kpos = 0xffffffffu;
        kq = QLO;
#pragma unroll
        for (int q = QLO; q < R; ++q) {
            if (!done[q]) {
                const unsigned kk = __float_as_uint(fabsf(p[q][j])) + 1u;
                if (kk > key || (kk == key && (unsigned)pos[q] < kpos)) {
                    key = kk;
                    kpos = pos[q];
                    kq = q;
                }
            }
        }
    };
    // Software pipeline: column j+1 is updated first and its reduction is
    // issued before the rest of column j's update, which hides its latency.
    unsigned key, kpos, kmax;
    int kq;
    candidate(0, key, kpos, kq);
    kmax = __reduce_max_sync(GLASS_FULL_MASK, key);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int cj = c0 + j;
        if (cj < n) {
            unsigned tie = __ballot_sync(GLASS_FULL_MASK, key == kmax);
            if (__popc(tie) > 1) {
                const unsigned pmin = __reduce_min_sync(GLASS_FULL_MASK, key == kmax ? kpos : 0xffffffffu);
                tie = __ballot_sync(GLASS_FULL_MASK, key == kmax && kpos == pmin);
            }
            const int wl = __ffs(tie) - 1;
            const unsigned packed = __shfl_sync(GLASS_FULL_MASK, (kpos << 4) | (unsigned)kq, wl);
            const int ppos = (int)(packed >> 4), wq = (int)(packed & 15u);
#pragma unroll
            for (int q = QLO; q < R; ++q) {
                if (pos[q] == cj) pos[q] = ppos;
                if (q == wq && lane == wl) {
                    pos[q] = cj;
                    done[q] = true;
                }
            }
            float sel = p[QLO][j];
#pragma unroll
            for (int q = QLO + 1; q < R; ++q)
                if (wq == q) sel = p[q][j];
            const float pv = __shfl_sync(GLASS_FULL_MASK, sel, wl);
            // a zero pivot (every candidate is zero) records info and eliminates
            // nothing: rc = 0 makes the multipliers and the update vanish
            const float rc = pv != 0.f ? __frcp_rn(pv) : 0.f;  // the correctly rounded 1 / pv
            if (lane == 0) {
                ipiv_s[cj] = ppos;
                dv[cj] = rc;
            }
            if (pv == 0.f && info == 0) info = cj + 1;
            float m[R];
#pragma unroll
            for (int q = QLO; q < R; ++q) {
                m[q] = p[q][j] * rc;
                if (!done[q]) p[q][j] = m[q];
            }
            auto update = [&](int k) {
                float s = p[QLO][k];
#pragma unroll
                for (int q = QLO + 1; q < R; ++q)
                    if (wq == q) s = p[q][k];
                const float pk = __shfl_sync(GLASS_FULL_MASK, s, wl);
#pragma unroll
                for (int q = QLO; q < R; ++q)
                    if (!done[q]) p[q][k] = fmaf(-m[q], pk, p[q][k]);
            };
            if (j + 1 < 16) {
                update(j + 1);
                if (cj + 1 < n) {
                    candidate(j + 1, key, kpos, kq);
                    kmax = __reduce_max_sync(GLASS_FULL_MASK, key);
                }
            }
#pragma unroll
            for (int k = 0; k < 16; ++k)  // fixed range: keeps p[][] in registers
                if (k > j + 1) update(k);
        }
    }
    if (c0 == 0) tcwarp::wait_all();  // columns 16.. of a stage_async'd operand
    // ---- 2. panel to its logical rows; permute the other columns and prow
    int pr[R];
#pragma unroll
    for (int q = QLO; q < R; ++q) pr[q] = prow[lane + 32 * q];
    __syncwarp();
    float *wp = opaque(As);
#pragma unroll
    for (int q = QLO; q < R; ++q) {
        const int row = lane + 32 * q;
        if (row >= c0 && row < n) {
#pragma unroll
            for (int k = 0; k < 16; ++k) wp[(c0 + k) * LD + pos[q]] = p[q][k];
            prow[pos[q]] = pr[q];
        }
    }
    for (int cb = 0; cb < n; cb += 16) {
        if (cb == c0) continue;
        float v[R][16];
#pragma unroll
        for (int q = QLO; q < R; ++q)
#pragma unroll
            for (int k = 0; k < 16; ++k) v[q][k] = As[(cb + k) * LD + lane + 32 * q];
        __syncwarp();
#pragma unroll
        for (int q = QLO; q < R; ++q) {
            const int row = lane + 32 * q;
            if (row >= c0 && row < n && pos[q] != row)
#pragma unroll
                for (int k = 0; k < 16; ++k) wp[(cb + k) * LD + pos[q]] = v[q][k];
        }
        __syncwarp();
    }
    __syncwarp();
}

// In-place LU of As (order n <= NMAX).  prow[i] (initially i) receives the
// original row held by logical row i; ipiv_s the interchanges, dv[j] = 1/u_jj.
// As may still be arriving from stage_async beyond column 15 (wait_first()
// done): the first panel factors columns 0..15 in registers and waits for
// the copies before it touches any other column.
template <int NMAX>
__device__ __forceinline__ int getrf(float *As, int n, int *prow, int *ipiv_s, float *dv) {
    constexpr int LD = Shape<NMAX>::LD;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    int info = 0;
    for (int c0 = 0; c0 < n; c0 += 16) {
        if constexpr (NMAX > 32) {
            if (c0 < 32) panel<NMAX, 0>(As, prow, n, c0, ipiv_s, dv, info);
            else panel<NMAX, 1>(As, prow, n, c0, ipiv_s, dv, info);
        } else {
            panel<NMAX, 0>(As, prow, n, c0, ipiv_s, dv, info);
        }
        float *wp = opaque(As);
        // ---- 3. U12 = L11^{-1} A12, one column per lane
        for (int c = c0 + 16 + lane; c < n; c += 32) {
            float x[16];
            const float4 *src = reinterpret_cast<const float4 *>(As + c * LD + c0);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 v4 = src[r];
                x[4 * r] = v4.x;
                x[4 * r + 1] = v4.y;
                x[4 * r + 2] = v4.z;
                x[4 * r + 3] = v4.w;
            }
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const float *lcol = As + (c0 + r) * LD + c0;
#pragma unroll
                for (int s = 0; s < 16; ++s)
                    if (s > r) x[s] = fmaf(-lcol[s], x[r], x[s]);
            }
            float4 *dst = reinterpret_cast<float4 *>(wp + c * LD + c0);
#pragma unroll
            for (int r = 0; r < 4; ++r) dst[r] = make_float4(x[4 * r], x[4 * r + 1], x[4 * r + 2], x[4 * r + 3]);
        }
        __syncwarp();
        // ---- 4. A22 -= L21 U12 on the tensor cores, 16 x 16 per step
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
            for (int C0 = r0; C0 < n; C0 += 16) {
                const bool two = C0 + 8 < n;
                float *c = wp + (C0 + 2 * t) * LD + R0 + g;
                float a0[4] = {c[0], c[LD], c[8], c[LD + 8]};
                float a1[4] = {0.f, 0.f, 0.f, 0.f};
                if (two) {
                    a1[0] = c[8 * LD];
                    a1[1] = c[9 * LD];
                    a1[2] = c[8 * LD + 8];
                    a1[3] = c[9 * LD + 8];
                }
                const float *u0 = As + (C0 + g) * LD + c0;
                const float *u1 = u0 + 8 * LD;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    unsigned bh0[2], bl0[2], bh1[2], bl1[2];
                    split(u0[8 * kk + t], bh0[0], bl0[0]);
                    split(u0[8 * kk + t + 4], bh0[1], bl0[1]);
                    split(u1[8 * kk + t], bh1[0], bl1[0]);
                    split(u1[8 * kk + t + 4], bh1[1], bl1[1]);
                    mma_tf32(a0, al[kk], bh0);
                    mma_tf32(a1, al[kk], bh1);
                    mma_tf32(a0, ah[kk], bl0);
                    mma_tf32(a1, ah[kk], bl1);
                    mma_tf32(a0, ah[kk], bh0);
                    mma_tf32(a1, ah[kk], bh1);
                }
                c[0] = a0[0];
                c[LD] = a0[1];
                c[8] = a0[2];
                c[LD + 8] = a0[3];
                if (two) {
                    c[8 * LD] = a1[0];
                    c[9 * LD] = a1[1];
                    c[8 * LD + 8] = a1[2];
                    c[9 * LD + 8] = a1[3];
                }
            }
        }
        __syncwarp();
    }
    return info;
}

// One right-hand side already gathered into logical row order (x[q] = row
// lane + 32q of P b): unit-lower forward and column-oriented upper backward
// sweeps against the packed factor, for 16 < n <= NMAX.  Each half of the
// rows is a fully unrolled loop with the pivot's lane and register slot
// known at compile time, so a step is one shuffle and one fused
// multiply-add per slot, and the column loads do not wait on the chain.
template <int NMAX>
__device__ __forceinline__ void getrs(const float *As, const float *dv, float (&x)[Shape<NMAX>::R], int n) {
    static_assert(NMAX == 32 || NMAX == 64, "orders 17..32 or 33..64");
    constexpr int LD = Shape<NMAX>::LD;
    const int lane = threadIdx.x & 31;
    if constexpr (NMAX == 32) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (i < n) {
                const float yi = __shfl_sync(GLASS_FULL_MASK, x[0], i);
                const float c0 = As[i * LD + lane];
                if (lane > i) x[0] = fmaf(-c0, yi, x[0]);
            }
        }
#pragma unroll
        for (int i = 31; i >= 0; --i) {
            if (i < n) {
                const float xi = __shfl_sync(GLASS_FULL_MASK, x[0], i) * dv[i];
                const float c0 = As[i * LD + lane];
                if (lane == i) x[0] = xi;
                else if (lane < i) x[0] = fmaf(-c0, xi, x[0]);
            }
        }
        return;
    } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) {  // rows 0..31 hold the pivots (n > 32)
        const float yi = __shfl_sync(GLASS_FULL_MASK, x[0], i);
        const float c0 = As[i * LD + lane], c1 = As[i * LD + lane + 32];
        if (lane > i) x[0] = fmaf(-c0, yi, x[0]);
        x[1] = fmaf(-c1, yi, x[1]);  // rows >= n: zero factor rows keep x = 0
    }
#pragma unroll
    for (int i = 32; i < 64; ++i) {
        if (i < n) {
            const float yi = __shfl_sync(GLASS_FULL_MASK, x[1], i - 32);
            const float c1 = As[i * LD + lane + 32];
            if (lane + 32 > i) x[1] = fmaf(-c1, yi, x[1]);
        }
    }
#pragma unroll
    for (int i = 63; i >= 32; --i) {
        if (i < n) {
            const float xi = __shfl_sync(GLASS_FULL_MASK, x[1], i - 32) * dv[i];
            const float c0 = As[i * LD + lane], c1 = As[i * LD + lane + 32];
            if (lane + 32 == i) x[1] = xi;
            else if (lane + 32 < i) x[1] = fmaf(-c1, xi, x[1]);
            x[0] = fmaf(-c0, xi, x[0]);
        }
    }
#pragma unroll
    for (int i = 31; i >= 0; --i) {
        const float xi = __shfl_sync(GLASS_FULL_MASK, x[0], i) * dv[i];
        const float c0 = As[i * LD + lane];
        if (lane == i) x[0] = xi;
        else if (lane < i) x[0] = fmaf(-c0, xi, x[0]);
    }
    }
}

}  // namespace tclu
}  // namespace glass
