// dev_chol_tc.cuh -- warp-scope blocked Cholesky with tensor-core trailing
// updates, for orders 17..64 (NMAX 32 or 64).
//
// One warp owns one problem held in its shared memory, column-major with
// pitch LD = NMAX + 8 (LD = 8 mod 32: every TF32 fragment load of the MMA
// touches 32 distinct banks).  The factorization runs over 16-column panels:
//   1. panel: the 16 columns c0..c0+15 (rows c0..n-1) are factored on the
//      SIMT pipe in registers (row i in lane i % 32), right-looking, with
//      the same diagonal rules as every other scope (Sec. III-B
//      factorizations; LAPACK info);
//   2. trailing update A22 -= L21 L21^T on the tensor cores: mma.sync
//      m16n8k8 TF32 over the 16x16 tiles of A22 that meet its lower
//      triangle (two independent 16x8 accumulators), each product split
//      3xTF32 (a = a_hi + a_lo; hi*hi + hi*lo + lo*hi) so the update keeps
//      FP32-level accuracy; FP32 accumulation.
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

// The sign bit flipped, as an instruction at each call (kept out of common
// subexpressions, so the result is not held in a register between uses).
__device__ __forceinline__ unsigned negate_bits(unsigned x) {
    unsigned r;
    asm volatile("xor.b32 %0, %1, 0x80000000;" : "=r"(r) : "r"(x));
    return r;
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

// Stage the column-major n x n operand at ga (leading dimension lda) into As
// (pitch LD, a multiple of 4) with cp.async copies, every copy of the lane
// in flight at once: 16-byte copies when n and lda are multiples of 4 and ga
// is 16-byte aligned, 4-byte copies otherwise.  Everything outside the
// operand is zero; LOWER skips what lies above the diagonal (16-byte groups
// wholly above it in the vector form) and leaves it zero or as read -- it is
// never used.  The copies form two groups, columns 0..15 first, so that a
// factorization can start on its first panel while the rest arrives: after
// stage_async, wait_first() makes columns 0..15 complete and visible to the
// warp, wait_all() everything.
template <int NMAX, bool LOWER, int LD = Shape<NMAX>::LD>
__device__ __forceinline__ void stage_async(float *As, const float *ga, long long lda, int n) {
    constexpr int R = Shape<NMAX>::R;
    const int lane = threadIdx.x & 31;
    const bool vec = (n & 3) == 0 && (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(ga) & 15) == 0;
    if (vec && n == NMAX && lda == NMAX) {
        // A full, packed problem: lane l copies 16-byte group l % G of
        // column l / G and every (32 / G)-th column after it, so each copy
        // is one instruction at a fixed offset from two base addresses.
        constexpr int G = NMAX / 4, CS = 32 / G, IT = NMAX / CS;
        const int k0 = lane / G, r = 4 * (lane % G);
        const float *src = ga + k0 * NMAX + r;
        float *dst = As + k0 * LD + r;
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            if (!LOWER || r + 3 >= k0 + CS * it) cp_async16(dst + CS * it * LD, src + CS * it * NMAX);
            else *reinterpret_cast<float4 *>(dst + CS * it * LD) = make_float4(0.f, 0.f, 0.f, 0.f);
            if (it == 16 / CS - 1) asm volatile("cp.async.commit_group;" ::: "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        return;
    }
    auto columns = [&](int k0, int k1) {
        if (vec) {
#pragma unroll 4
            for (int e = k0 * (NMAX / 4) + lane; e < k1 * (NMAX / 4); e += 32) {
                const int k = e / (NMAX / 4), r = 4 * (e % (NMAX / 4));
                float *d = As + k * LD + r;
                if (k < n && r < n && (!LOWER || r + 3 >= k)) cp_async16(d, ga + (long long)k * lda + r);
                else *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
#pragma unroll 4
            for (int k = k0; k < k1; ++k)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int i = lane + 32 * q;
                    float *d = As + k * LD + i;
                    if (k < n && i < n && (!LOWER || i >= k)) cp_async4(d, ga + (long long)k * lda + i);
                    else *d = 0.f;
                }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    columns(0, 16);
    columns(16, NMAX);
}
__device__ __forceinline__ void wait_first() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();
}
__device__ __forceinline__ void wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
}

// stage_async, then everything complete and visible to the warp.
template <int NMAX, bool LOWER, int LD = Shape<NMAX>::LD>
__device__ __forceinline__ void stage(float *As, const float *ga, long long lda, int n) {
    stage_async<NMAX, LOWER, LD>(As, ga, lda, n);
    wait_all();
}

// Write the n x n result in As back to ga (LOWER: the lower triangle only,
// the rest of ga keeps its contents), 16-byte stores where whole 16-byte
// groups are written and the operand is aligned as for stage().
template <int NMAX, bool LOWER, int LD = Shape<NMAX>::LD>
__device__ __forceinline__ void unstage(float *ga, long long lda, const float *As, int n) {
    constexpr int R = Shape<NMAX>::R;
    const int lane = threadIdx.x & 31;
    const bool vec = (n & 3) == 0 && (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(ga) & 15) == 0;
    float *wg = opaque(ga);
    if (vec && n == NMAX && lda == NMAX) {  // the lane-to-group map of stage_async's full form
        constexpr int G = NMAX / 4, CS = 32 / G, IT = NMAX / CS;
        const int k0 = lane / G, r = 4 * (lane % G);
        float *dst = wg + k0 * NMAX + r;
        const float *src = As + k0 * LD + r;
#pragma unroll
        for (int it = 0; it < IT; ++it) {  // LOWER: the groups wholly on or below the diagonal
            const float4 v = *reinterpret_cast<const float4 *>(src + CS * it * LD);
            if (!LOWER || r >= k0 + CS * it) __stcs(reinterpret_cast<float4 *>(dst + CS * it * NMAX), v);
        }
        if constexpr (LOWER) {
            // The rest of the lower triangle: in each 4 x 4 diagonal block
            // (first row and column 4c), the six entries (4c + i, 4c + j)
            // with 1 <= j <= i <= 3, numbered w = 0..5 column by column.
#pragma unroll
            for (int e = lane; e < 6 * (NMAX / 4); e += 32) {
                const int c = e / 6, w = e - 6 * c;
                const int j = w < 3 ? 1 : (w < 5 ? 2 : 3);
                const int i = w < 3 ? w + 1 : (w < 5 ? w - 1 : 3);
                const int row = 4 * c + i, col = 4 * c + j;
                wg[col * NMAX + row] = As[col * LD + row];
            }
        }
        return;
    }
    if (vec) {
#pragma unroll 4
        for (int e = lane; e < NMAX * NMAX / 4; e += 32) {
            const int k = e / (NMAX / 4), r = 4 * (e % (NMAX / 4));
            if (k >= n || r >= n || (LOWER && r + 3 < k)) continue;
            const float4 v = *reinterpret_cast<const float4 *>(As + k * LD + r);
            float *d = wg + (long long)k * lda + r;
            if (!LOWER || r >= k) {
                __stcs(reinterpret_cast<float4 *>(d), v);
            } else {  // the group holding the diagonal
                if (r >= k) d[0] = v.x;
                if (r + 1 >= k) d[1] = v.y;
                if (r + 2 >= k) d[2] = v.z;
                d[3] = v.w;
            }
        }
    } else {
#pragma unroll 4
        for (int k = 0; k < NMAX; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (k < n && i < n && (!LOWER || i >= k)) wg[(long long)k * lda + i] = As[k * LD + i];
            }
    }
}

// Panel c0 of the factorization (rows held in slots q >= QLO; the slots
// below hold rows above the panel only), right-looking in registers.  Per
// column the raw entries of rows c0..c0+15 are published to a 16-float
// shared segment (two, alternating) and read back by every lane as 16-byte
// broadcasts: the pivot comes from there, and with u_i = l_ij / l_jj formed
// once per row the update of column k is one fused multiply-add per row
// (a_ik -= u_i a_kj).  Rows above the diagonal are updated too -- their
// values are never read and never written back.  The lower part is written
// back and mirrored, transposed, into the unused upper triangle
// (As[i * LD + r] = l_ir for r < i), where the backward solve reads rows of
// L as contiguous columns.
template <int NMAX, int QLO>
__device__ __forceinline__ void panel(float *As, int n, int c0, float *dv, float *bc, bool fp64diag, int &info) {
    constexpr int LD = Shape<NMAX>::LD;
    constexpr int R = Shape<NMAX>::R;
    const int lane = threadIdx.x & 31;
    float p[R][16];
#pragma unroll
    for (int q = QLO; q < R; ++q)
#pragma unroll
        for (int k = 0; k < 16; ++k) p[q][k] = As[(c0 + k) * LD + lane + 32 * q];
    // rows c0..c0+15 of column j go to segment j & 1
    auto publish = [&](int j) {
        float *buf = bc + 16 * (j & 1);
#pragma unroll
        for (int q = QLO; q < R; ++q) {
            const int i = lane + 32 * q;
            if (i >= c0 && i < c0 + 16) buf[i - c0] = p[q][j];
        }
    };
    // Software pipeline: column j+1 is updated and published before the
    // rest of column j's update, which hides the publish latency.
    publish(0);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int cj = c0 + j;
        if (cj < n) {
            __syncwarp();
            float s[16];
            {
                const float4 *b4 = reinterpret_cast<const float4 *>(bc + 16 * (j & 1));
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float4 v = b4[m];
                    s[4 * m] = v.x;
                    s[4 * m + 1] = v.y;
                    s[4 * m + 2] = v.z;
                    s[4 * m + 3] = v.w;
                }
            }
            const float d = s[j];
            if (!(d > 0.f) && info == 0) info = cj + 1;
            float l, r;
            chol_diag(d, fp64diag, l, r);
            if (lane == 0) dv[cj] = r;
            // u_i = l_ij / l_jj, so that l_ij l_kj = u_i a_kj: one fused
            // multiply-add per entry of the update, no product per column.
            float u[R];
#pragma unroll
            for (int q = QLO; q < R; ++q) {
                p[q][j] = (lane + 32 * q == cj) ? l : p[q][j] * r;
                u[q] = p[q][j] * r;
            }
            if (j + 1 < 16) {
#pragma unroll
                for (int q = QLO; q < R; ++q) p[q][j + 1] = fmaf(-u[q], s[j + 1], p[q][j + 1]);
                publish(j + 1);
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {  // fixed range: keeps p[][] in registers
                if (k > j + 1) {
#pragma unroll
                    for (int q = QLO; q < R; ++q) p[q][k] = fmaf(-u[q], s[k], p[q][k]);
                }
            }
        }
    }
    float *wp = opaque(As);
#pragma unroll
    for (int q = QLO; q < R; ++q) {
        const int i = lane + 32 * q;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (i >= c0 + k && i < n) wp[(c0 + k) * LD + i] = p[q][k];
        if (i >= c0 + 16 && i < n) {
            float4 *dst = reinterpret_cast<float4 *>(wp + i * LD + c0);
#pragma unroll
            for (int k = 0; k < 4; ++k) dst[k] = make_float4(p[q][4 * k], p[q][4 * k + 1], p[q][4 * k + 2], p[q][4 * k + 3]);
        } else if (i > c0 && i < n) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (c0 + k < i) wp[i * LD + c0 + k] = p[q][k];
        }
    }
    __syncwarp();
}

// In-place Cholesky of the lower triangle of As (order n <= NMAX); dv[j]
// receives 1 / l_jj; bc is 32 floats (16-byte aligned) of per-warp scratch.
// As may still be arriving from stage_async beyond column 15 (wait_first()
// done): the first panel reads only columns 0..15, and the copies are
// waited for before anything else.  Returns info (uniform).
template <int NMAX>
__device__ __forceinline__ int potrf(float *As, int n, float *dv, float *bc, bool fp64diag) {
    constexpr int LD = Shape<NMAX>::LD;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    int info = 0;
    for (int c0 = 0; c0 < n; c0 += 16) {
        // ---- 1. panel on the SIMT pipe
        if constexpr (NMAX > 32) {
            if (c0 < 32) panel<NMAX, 0>(As, n, c0, dv, bc, fp64diag, info);
            else panel<NMAX, 1>(As, n, c0, dv, bc, fp64diag, info);
        } else {
            panel<NMAX, 0>(As, n, c0, dv, bc, fp64diag, info);
        }
        if (c0 == 0) wait_all();  // columns 16.. of a stage_async'd operand (a no-op after stage)
        // ---- 2. trailing update on the tensor cores, 16 x 16 per step.
        // Row tile rt of L21 is the A operand of the tiles in its row and,
        // transposed, the B operand of the tiles in column rt, with the same
        // per-lane entries: each is split once (sh/sl); the A operand is the
        // negated split (split(-x) = -split(x): TF32 rounding is symmetric).
        float *wp = opaque(As);
        const int r0 = c0 + 16;
        constexpr int NT = NMAX / 16 - 1;
        unsigned sh[NT][2][4], sl[NT][2][4];
#pragma unroll
        for (int rt = 0; rt < NT; ++rt) {  // fixed trip counts: the tiles interleave
            const int R0 = r0 + 16 * rt;
            if (R0 >= n) break;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const float *col = As + (c0 + 8 * kk + t) * LD;
                split(col[R0 + g], sh[rt][kk][0], sl[rt][kk][0]);
                split(col[R0 + g + 8], sh[rt][kk][1], sl[rt][kk][1]);
                split(col[4 * LD + R0 + g], sh[rt][kk][2], sl[rt][kk][2]);
                split(col[4 * LD + R0 + g + 8], sh[rt][kk][3], sl[rt][kk][3]);
            }
#pragma unroll
            for (int ct = 0; ct <= rt; ++ct) {
                const int C0 = r0 + 16 * ct;
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
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    unsigned ah[4], al[4];  // formed at each use: held for all tiles they would cost 16 registers
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        ah[e] = negate_bits(sh[rt][kk][e]);
                        al[e] = negate_bits(sl[rt][kk][e]);
                    }
                    const unsigned bh0[2] = {sh[ct][kk][0], sh[ct][kk][2]}, bl0[2] = {sl[ct][kk][0], sl[ct][kk][2]};
                    const unsigned bh1[2] = {sh[ct][kk][1], sh[ct][kk][3]}, bl1[2] = {sl[ct][kk][1], sl[ct][kk][3]};
                    mma_tf32(a0, al, bh0);
                    mma_tf32(a1, al, bh1);
                    mma_tf32(a0, ah, bl0);
                    mma_tf32(a1, ah, bl1);
                    mma_tf32(a0, ah, bh0);
                    mma_tf32(a1, ah, bh1);
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

// One right-hand side held like the rows (x[q] = row lane + 32q) against L
// in shared memory, for 16 < n <= NMAX: x <- L^{-1} x down the columns of L,
// then x <- L^{-T} x down the columns of the mirrored upper triangle.  Each
// half of the rows is a fully unrolled loop (the pivot's lane and slot known
// at compile time): one shuffle and one fused multiply-add per slot and step,
// column loads independent of the chain.
template <int NMAX>
__device__ __forceinline__ void potrs(const float *As, const float *dv, float (&x)[Shape<NMAX>::R], int n) {
    static_assert(NMAX == 32 || NMAX == 64, "orders 17..32 or 33..64");
    constexpr int LD = Shape<NMAX>::LD;
    const int lane = threadIdx.x & 31;
    // 1/l_ii of the lane's own rows (zero past n): step i multiplies in
    // lane i before the broadcast, so no step reads dv[i]
    float d[Shape<NMAX>::R];
#pragma unroll
    for (int q = 0; q < Shape<NMAX>::R; ++q) d[q] = lane + 32 * q < n ? dv[lane + 32 * q] : 0.f;
    if constexpr (NMAX == 32) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (i < n) {
                const float yi = __shfl_sync(GLASS_FULL_MASK, x[0] * d[0], i);
                const float c0 = As[i * LD + lane];
                if (lane == i) x[0] = yi;
                else if (lane > i) x[0] = fmaf(-c0, yi, x[0]);
            }
        }
#pragma unroll
        for (int i = 31; i >= 0; --i) {
            if (i < n) {
                const float xi = __shfl_sync(GLASS_FULL_MASK, x[0] * d[0], i);
                const float c0 = As[i * LD + lane];
                if (lane == i) x[0] = xi;
                else if (lane < i) x[0] = fmaf(-c0, xi, x[0]);
            }
        }
        return;
    } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float yi = __shfl_sync(GLASS_FULL_MASK, x[0] * d[0], i);
        const float c0 = As[i * LD + lane], c1 = As[i * LD + lane + 32];
        if (lane == i) x[0] = yi;
        else if (lane > i) x[0] = fmaf(-c0, yi, x[0]);
        x[1] = fmaf(-c1, yi, x[1]);  // rows >= n: zero factor rows keep x = 0
    }
#pragma unroll
    for (int i = 32; i < 64; ++i) {
        if (i < n) {
            const float yi = __shfl_sync(GLASS_FULL_MASK, x[1] * d[1], i - 32);
            const float c1 = As[i * LD + lane + 32];
            if (lane + 32 == i) x[1] = yi;
            else if (lane + 32 > i) x[1] = fmaf(-c1, yi, x[1]);
        }
    }
#pragma unroll
    for (int i = 63; i >= 32; --i) {
        if (i < n) {
            const float xi = __shfl_sync(GLASS_FULL_MASK, x[1] * d[1], i - 32);
            const float c0 = As[i * LD + lane], c1 = As[i * LD + lane + 32];  // mirror: l_{i,row}
            if (lane + 32 == i) x[1] = xi;
            else if (lane + 32 < i) x[1] = fmaf(-c1, xi, x[1]);
            x[0] = fmaf(-c0, xi, x[0]);
        }
    }
#pragma unroll
    for (int i = 31; i >= 0; --i) {
        const float xi = __shfl_sync(GLASS_FULL_MASK, x[0] * d[0], i);
        const float c0 = As[i * LD + lane];
        if (lane == i) x[0] = xi;
        else if (lane < i) x[0] = fmaf(-c0, xi, x[0]);
    }
    }
}

// K right-hand sides at once (x[k][q] = row lane + 32q of column k), the
// same sweeps as potrs with the K independent chains interleaved step by
// step: K shuffles and K fused multiply-adds per slot and step, so the
// latency of one shuffle-and-update chain is shared by K solves.
template <int NMAX, int K>
__device__ __forceinline__ void potrs_k(const float *As, const float *dv, float (&x)[K][Shape<NMAX>::R], int n) {
    static_assert(NMAX == 32 || NMAX == 64, "orders 17..32 or 33..64");
    constexpr int LD = Shape<NMAX>::LD;
    constexpr int R = Shape<NMAX>::R;
    const int lane = threadIdx.x & 31;
    // forward: x <- L^{-1} x down the columns of L
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i < n) {
            const int qi = i / 32, li = i % 32;
            const float d = dv[i];
            float c[R];
#pragma unroll
            for (int q = 0; q < R; ++q) c[q] = As[i * LD + lane + 32 * q];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float yi = __shfl_sync(GLASS_FULL_MASK, x[k][qi], li) * d;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = lane + 32 * q;
                    if (row == i) x[k][q] = yi;
                    else if (row > i) x[k][q] = fmaf(-c[q], yi, x[k][q]);  // rows >= n: zero factor rows
                }
            }
        }
    }
    // backward: x <- L^{-T} x down the columns of the mirrored upper triangle
#pragma unroll
    for (int i = NMAX - 1; i >= 0; --i) {
        if (i < n) {
            const int qi = i / 32, li = i % 32;
            const float d = dv[i];
            float c[R];
#pragma unroll
            for (int q = 0; q < R; ++q) c[q] = As[i * LD + lane + 32 * q];  // l_{i,row} for row < i
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float xi = __shfl_sync(GLASS_FULL_MASK, x[k][qi], li) * d;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int row = lane + 32 * q;
                    if (row == i) x[k][q] = xi;
                    else if (row < i) x[k][q] = fmaf(-c[q], xi, x[k][q]);
                }
            }
        }
    }
}

}  // namespace tcwarp
}  // namespace glass
