// dev_lu_tc2.cuh -- blocked LU with partial pivoting and tensor-core
// trailing updates for orders 33..64, run by a team of two warps per problem
// (the block-scope placement of those orders).
//
// The problem sits in the team's shared memory as in the one-warp form
// (dev_lu_tc.cuh: column-major, pitch 72, rows and columns beyond n zero),
// and the steps are the same -- per 16-column panel: the panel factored in
// registers with partial pivoting (largest |a|, smallest current row index
// on ties; rows never move inside the panel, only their logical positions
// change), the panel's permutation applied to every other column and to the
// record of original rows, U12 = L11^{-1} A12, A22 -= L21 U12 on 3xTF32
// mma.sync -- with the work of each step split over 64 threads:
//   - panel: row r belongs to lane r / 2 of warp r % 2, so both warps hold
//     live rows of every panel.  Per column each warp reduces its own
//     candidates, its winning lane publishes key, position and its whole
//     16-entry panel row to a double-buffered shared-memory slot, one named
//     barrier, and every thread reads both slots: the better candidate is
//     the pivot, and its row -- the multipliers' partners -- comes from
//     shared memory as four 16-byte broadcasts (no shuffle per column of
//     the update);
//   - interchanges: every thread moves its own row;
//   - U12: one column per thread;
//   - trailing update: the 16 x 16 tiles dealt alternately to the warps;
//   - after the factorization one warp solves while the other writes the
//     factor, the interchanges and info back.
// Every element sees the same operations in the same order as in the
// one-warp form, so the two produce identical results.
#pragma once

#include "dev_chol_tc.cuh"

namespace glass {
namespace tclu2 {

using tcwarp::mma_tf32;
using tcwarp::split;

constexpr int NMAX = 64;
constexpr int LD = NMAX + 8;  // 8 mod 32: conflict-free TF32 fragments
constexpr int T = 64;         // threads per team
constexpr int XS = 20;        // floats per exchange slot: 16 row entries, key, position (16-byte aligned)

// Shared-memory floats of one team: A, 1/u_jj, the interchanges, the
// original row of each logical row, and 2 parities x 2 warps exchange slots.
constexpr int floats() { return NMAX * LD + 3 * NMAX + 4 * XS; }

__device__ __forceinline__ void bar(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(T) : "memory"); }

// Stage the column-major n x n operand into As with cp.async over the team
// (16-byte copies when n and lda are multiples of 4 and ga is 16-byte
// aligned, 4-byte copies otherwise), zero elsewhere in the NMAX x NMAX
// block; complete and visible to the team on return.
__device__ __forceinline__ void stage(float *As, const float *ga, long long lda, int n, int rank, int bid) {
    const bool vec = (n & 3) == 0 && (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(ga) & 15) == 0;
    if (vec) {
        for (int e = rank; e < NMAX * NMAX / 4; e += T) {
            const int k = e >> 4, r = 4 * (e & 15);
            float *d = As + k * LD + r;
            if (k < n && r < n) cp_async16(d, ga + (long long)k * lda + r);
            else *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int e = rank; e < NMAX * NMAX; e += T) {
            const int k = e >> 6, i = e & 63;
            float *d = As + k * LD + i;
            if (k < n && i < n) cp_async4(d, ga + (long long)k * lda + i);
            else *d = 0.f;
        }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    bar(bid);
}

// In-place LU of As (order 32 < n <= 64) by the team: prow[i] (initially i)
// receives the original row held by logical row i, ipiv_s the interchanges
// in sequential form, dv[j] = 1/u_jj.  Returns info (uniform over the team).
__device__ __forceinline__ int getrf(float *As, int n, int *prow, int *ipiv_s, float *dv, float *xch, int rank,
                                     int bid) {
    const int w = rank >> 5, lane = rank & 31, g = lane >> 2, t = lane & 3;
    const int row = 2 * lane + w;
    int info = 0;
    float *wp = opaque(As);
    for (int c0 = 0; c0 < n; c0 += 16) {
        // ---- 1. panel: this thread's row in registers
        float p[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) p[k] = As[(c0 + k) * LD + row];
        int pos = row;
        bool done = row < c0 || row >= n;
        auto key_of = [&](int j) { return done ? 0u : __float_as_uint(fabsf(p[j])) + 1u; };
        unsigned key = key_of(0);
        unsigned kmax = __reduce_max_sync(GLASS_FULL_MASK, key);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int cj = c0 + j;
            if (cj < n) {
                // the warp's candidate: largest key, then smallest position
                unsigned tie = __ballot_sync(GLASS_FULL_MASK, key == kmax);
                unsigned wpos = (unsigned)pos;
                if (__popc(tie) > 1) {
                    const unsigned pmin = __reduce_min_sync(GLASS_FULL_MASK, key == kmax ? wpos : 0xffffffffu);
                    tie = __ballot_sync(GLASS_FULL_MASK, key == kmax && wpos == pmin);
                }
                const int wl = __ffs(tie) - 1;
                float *slots = xch + (j & 1) * 2 * XS;
                if (lane == wl) {
                    float4 *s4 = reinterpret_cast<float4 *>(slots + w * XS);
#pragma unroll
                    for (int m = 0; m < 4; ++m) s4[m] = make_float4(p[4 * m], p[4 * m + 1], p[4 * m + 2], p[4 * m + 3]);
                    slots[w * XS + 16] = __uint_as_float(kmax);
                    slots[w * XS + 17] = __int_as_float(pos);
                }
                bar(bid);
                // the team's pivot: the better of the two candidates
                const unsigned k0 = __float_as_uint(slots[16]), k1 = __float_as_uint(slots[XS + 16]);
                const int p0 = __float_as_int(slots[17]), p1 = __float_as_int(slots[XS + 17]);
                const int ww = (k1 > k0 || (k1 == k0 && p1 < p0)) ? 1 : 0;
                const int ppos = ww ? p1 : p0;
                float u[16];
                {
                    const float4 *s4 = reinterpret_cast<const float4 *>(slots + ww * XS);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const float4 v = s4[m];
                        u[4 * m] = v.x;
                        u[4 * m + 1] = v.y;
                        u[4 * m + 2] = v.z;
                        u[4 * m + 3] = v.w;
                    }
                }
                if (pos == cj) pos = ppos;
                if (w == ww && lane == wl) {
                    pos = cj;
                    done = true;
                }
                const float pv = u[j];
                // a zero pivot (every candidate is zero) records info and eliminates
                // nothing: rc = 0 makes the multipliers and the update vanish
                const float rc = pv != 0.f ? __frcp_rn(pv) : 0.f;  // the correctly rounded 1 / pv
                if (rank == 0) {
                    ipiv_s[cj] = ppos;
                    dv[cj] = rc;
                }
                if (pv == 0.f && info == 0) info = cj + 1;
                const float m = p[j] * rc;
                if (!done) p[j] = m;
                // column j+1 first, and its reduction issued before the rest
                if (j + 1 < 16) {
                    if (!done) p[j + 1] = fmaf(-m, u[j + 1], p[j + 1]);
                    if (cj + 1 < n) {
                        key = key_of(j + 1);
                        kmax = __reduce_max_sync(GLASS_FULL_MASK, key);
                    }
                }
#pragma unroll
                for (int k = 0; k < 16; ++k)  // fixed range: keeps p[] in registers
                    if (k > j + 1 && !done) p[k] = fmaf(-m, u[k], p[k]);
            }
        }
        // ---- 2. panel to its logical rows; permute the other columns and prow
        const int pr = prow[row];
        bar(bid);
        if (row >= c0 && row < n) {
#pragma unroll
            for (int k = 0; k < 16; ++k) wp[(c0 + k) * LD + pos] = p[k];
            prow[pos] = pr;
        }
        for (int cb = 0; cb < n; cb += 16) {
            if (cb == c0) continue;
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = As[(cb + k) * LD + row];
            bar(bid);
            if (row >= c0 && row < n && pos != row)
#pragma unroll
                for (int k = 0; k < 16; ++k) wp[(cb + k) * LD + pos] = v[k];
        }
        bar(bid);
        // ---- 3. U12 = L11^{-1} A12, one column per thread
        for (int c = c0 + 16 + rank; c < n; c += T) {
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
        bar(bid);
        // ---- 4. A22 -= L21 U12 on the tensor cores, the 16 x 16 tiles dealt
        // alternately to the two warps
        const int r0 = c0 + 16;
        const int nt = (n - r0 + 15) / 16;  // tiles per side of A22 (0 after the last panel)
        for (int tile = w; tile < nt * nt; tile += 2) {
            const int R0 = r0 + 16 * (tile / nt), C0 = r0 + 16 * (tile % nt);
            unsigned ah[2][4], al[2][4];
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const float *col = As + (c0 + 8 * kk + t) * LD;
                split(-col[R0 + g], ah[kk][0], al[kk][0]);
                split(-col[R0 + g + 8], ah[kk][1], al[kk][1]);
                split(-col[4 * LD + R0 + g], ah[kk][2], al[kk][2]);
                split(-col[4 * LD + R0 + g + 8], ah[kk][3], al[kk][3]);
            }
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
        bar(bid);
    }
    return info;
}

}  // namespace tclu2
}  // namespace glass
