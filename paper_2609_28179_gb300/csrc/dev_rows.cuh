// dev_rows.cuh -- block-scope ("row team") primitives: a team of T = 64
// threads owns one problem of order n <= NMAX <= 64, thread i holding row i
// of the operand in registers.  Values another row needs -- the current
// column of a Cholesky step, the pivot row of an LU step, a solved
// component -- go through the team's shared scratch, read back as 16-byte
// broadcasts, with the team's named barrier between producer and consumer.
// Same conventions as every other scope (Sec. III-A): lower factor, LAPACK
// info, sequential-swap ipiv, partial pivoting with the smallest row index
// on ties.
//
// Team scratch (floats, 16-byte aligned), `RS` right-hand sides per pass:
//   col[2][NMAX + 4]  double-buffered column / pivot row
//   dv[NMAX]          1 / l_jj  or  1 / u_jj
//   pp[NMAX]          pivot physical row per step (LU)
//   xb[2][RS*4]       double-buffered broadcast of solved components
//   red[2][2][RS]     per-warp partial sums (two buffers)
//   key[2][4]         per-warp pivot candidates
#pragma once

#include "common.cuh"

namespace glass {
namespace rows {

constexpr int T = 64;  // threads per team

template <int NMAX, int RS>
struct Scratch {
    static constexpr int COL = NMAX + 4;
    static constexpr int floats = 2 * COL + NMAX + NMAX + 2 * RS * 4 + 4 * RS + 8;
    float *col0, *col1, *dv, *xb0, *xb1, *red;
    int *pp, *key;
    __device__ Scratch(float *base) {
        col0 = base;
        col1 = base + COL;
        dv = base + 2 * COL;
        pp = reinterpret_cast<int *>(dv + NMAX);
        xb0 = dv + 2 * NMAX;
        xb1 = xb0 + RS * 4;
        red = xb1 + RS * 4;
        key = reinterpret_cast<int *>(red + 4 * RS);
    }
};

__device__ __forceinline__ void bar(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(T) : "memory"); }

// ------------------------------------------------------------- Cholesky
// a[0..NMAX): row i (k <= i meaningful).  Right-looking; at the start of
// step j the raw column j (rows >= j) is published in col[j & 1].  Every
// thread forms 1/l_jj itself, so one barrier per step suffices.
template <int NMAX, int RS>
__device__ __forceinline__ int potrf(float (&a)[NMAX], int n, int i, bool fp64diag, Scratch<NMAX, RS> &s, int bid) {
    int info = 0;
    if (i < n) s.col0[i] = a[0];
    bar(bid);
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            const float *cj = (j & 1) ? s.col1 : s.col0;
            float *cn = (j & 1) ? s.col0 : s.col1;
            const float d = cj[j];
            if (!(d > 0.f) && info == 0) info = j + 1;
            float l, r;
            chol_diag(d, fp64diag, l, r);
            if (i == j) { a[j] = l; s.dv[j] = r; }
            if (i > j && i < n) {
                const float lij = a[j] * r;
                a[j] = lij;
                const float sc = lij * r;
#pragma unroll
                for (int k4 = (j + 1) / 4; k4 < (NMAX + 3) / 4; ++k4) {
                    const float4 v = *reinterpret_cast<const float4 *>(cj + 4 * k4);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = 4 * k4 + u;
                        if (k > j && k < NMAX && k <= i) a[k] = fmaf(-sc, vv[u], a[k]);
                    }
                    // bound how far ahead the compiler hoists the broadcasts
                    // (each one holds four registers until used)
                    if ((k4 & 3) == 3) asm volatile("" ::: "memory");
                }
            }
            if constexpr (NMAX > 1) {
                if (j + 1 < NMAX && i > j && i < n) cn[i] = a[(j + 1) < NMAX ? j + 1 : j];
            }
            bar(bid);
        }
    }
    return info;
}

// x[0..RS) (rows i of RS right-hand sides) <- L^{-1} x: at step j thread j
// publishes y_j, then every row below takes -l_ij y_j.
template <int NMAX, int RS>
__device__ __forceinline__ void forward(const float (&a)[NMAX], float (&x)[RS], int n, int i, Scratch<NMAX, RS> &s,
                                        int bid) {
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            float *xb = (j & 1) ? s.xb1 : s.xb0;
            if (i == j) {
#pragma unroll
                for (int c = 0; c < RS; ++c) { x[c] *= s.dv[j]; xb[c] = x[c]; }
            }
            bar(bid);
            if (i > j && i < n) {
#pragma unroll
                for (int c = 0; c < RS; ++c) x[c] = fmaf(-a[j], xb[c], x[c]);
            }
        }
    }
}

// x <- L^{-T} x: x_j = (y_j - sum_{k>j} l_kj x_k) / l_jj; thread k holds
// l_kj, the sum is a warp reduction plus one shared exchange per step.
template <int NMAX, int RS>
__device__ __forceinline__ void backward_t(const float (&a)[NMAX], float (&x)[RS], int n, int i, Scratch<NMAX, RS> &s,
                                           int bid) {
    const int w = (threadIdx.x >> 5) & 1, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = NMAX - 1; j >= 0; --j) {
        if (j < n) {
            float *red = s.red + (j & 1) * 2 * RS;
#pragma unroll
            for (int c = 0; c < RS; ++c) {
                const float p = warp_sum((i > j && i < n) ? a[j] * x[c] : 0.f);
                if (lane == 0) red[w * RS + c] = p;
            }
            bar(bid);
            if (i == j) {
#pragma unroll
                for (int c = 0; c < RS; ++c) x[c] = (x[c] - (red[c] + red[RS + c])) * s.dv[j];
            }
        }
    }
}

// ------------------------------------------------------------------- LU
// Thread i holds PHYSICAL row i for the whole factorization; pos = its
// current logical position.  Step j: team argmax (warp redux, then the two
// warps' candidates through shared memory), the winner publishes its row,
// every remaining row eliminates.  ipiv_out[j] (global) gets the logical
// position of the winner.  Returns info.
template <int NMAX, int RS>
__device__ __forceinline__ int getrf(float (&a)[NMAX], int &pos, bool &done, int n, int i, Scratch<NMAX, RS> &s,
                                     int *ipiv_out, int bid) {
    const int w = (threadIdx.x >> 5) & 1, lane = threadIdx.x & 31;
    int info = 0;
    pos = i;
    done = false;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        if (j < n) {
            const bool cand = !done && i < n;
            const unsigned key = cand ? __float_as_uint(fabsf(a[j])) + 1u : 0u;
            const unsigned kmax = __reduce_max_sync(GLASS_FULL_MASK, key);
            const unsigned kpos = __reduce_min_sync(GLASS_FULL_MASK, (key == kmax && cand) ? (unsigned)pos : 0xffffffffu);
            int *kb = s.key + (j & 1) * 4;
            if (lane == 0) { kb[2 * w] = (int)kmax; kb[2 * w + 1] = (int)kpos; }
            bar(bid);
            const unsigned k0 = (unsigned)kb[0], k1 = (unsigned)kb[2];
            const unsigned p0 = (unsigned)kb[1], p1 = (unsigned)kb[3];
            const int ppos = (int)((k0 > k1 || (k0 == k1 && p0 < p1)) ? p0 : p1);
            const bool winner = cand && pos == ppos;
            float *prow = (j & 1) ? s.col1 : s.col0;
            if (winner) {
                s.pp[j] = i;
#pragma unroll
                for (int k4 = j / 4; k4 < (NMAX + 3) / 4; ++k4) {
                    float4 v;
                    v.x = 4 * k4 + 0 < NMAX ? a[(4 * k4 + 0) < NMAX ? 4 * k4 + 0 : 0] : 0.f;
                    v.y = 4 * k4 + 1 < NMAX ? a[(4 * k4 + 1) < NMAX ? 4 * k4 + 1 : 0] : 0.f;
                    v.z = 4 * k4 + 2 < NMAX ? a[(4 * k4 + 2) < NMAX ? 4 * k4 + 2 : 0] : 0.f;
                    v.w = 4 * k4 + 3 < NMAX ? a[(4 * k4 + 3) < NMAX ? 4 * k4 + 3 : 0] : 0.f;
                    *reinterpret_cast<float4 *>(prow + 4 * k4) = v;
                }
            }
            if (threadIdx.x % T == 0 && ipiv_out != nullptr) ipiv_out[j] = ppos;
            bar(bid);
            if (pos == j) pos = ppos;
            if (winner) { pos = j; done = true; }
            const float pv = prow[j];
            const float rc = pv != 0.f ? 1.0f / pv : 0.f;
            if (i == 0) s.dv[j] = rc;
            if (pv == 0.f) {
                if (info == 0) info = j + 1;
                continue;
            }
            if (!done && i < n) {
                const float m = a[j] * rc;
                a[j] = m;
#pragma unroll
                for (int k4 = (j + 1) / 4; k4 < (NMAX + 3) / 4; ++k4) {
                    const float4 v = *reinterpret_cast<const float4 *>(prow + 4 * k4);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = 4 * k4 + u;
                        if (k > j && k < NMAX) a[k] = fmaf(-m, vv[u], a[k]);
                    }
                    if ((k4 & 3) == 3) asm volatile("" ::: "memory");
                }
            }
        }
    }
    bar(bid);
    return info;
}

// x[0..RS) = b of this thread's ORIGINAL row i; on return x is the solution
// component at logical position pos.
template <int NMAX, int RS>
__device__ __forceinline__ void getrs(const float (&a)[NMAX], int pos, float (&x)[RS], int n, int i,
                                      Scratch<NMAX, RS> &s, int bid) {
    bar(bid);  // earlier readers of the broadcast buffers are done
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {  // unit lower, logical order
        if (j < n) {
            float *xb = (j & 1) ? s.xb1 : s.xb0;
            if (i == s.pp[j])
#pragma unroll
                for (int c = 0; c < RS; ++c) xb[c] = x[c];
            bar(bid);
            if (pos > j && i < n)
#pragma unroll
                for (int c = 0; c < RS; ++c) x[c] = fmaf(-a[j], xb[c], x[c]);
        }
    }
    bar(bid);  // the forward sweep's last broadcast has been read
#pragma unroll
    for (int j = NMAX - 1; j >= 0; --j) {  // upper, logical order
        if (j < n) {
            float *xb = (j & 1) ? s.xb1 : s.xb0;
            if (i == s.pp[j])
#pragma unroll
                for (int c = 0; c < RS; ++c) { x[c] *= s.dv[j]; xb[c] = x[c]; }
            bar(bid);
            if (pos < j && i < n)
#pragma unroll
                for (int c = 0; c < RS; ++c) x[c] = fmaf(-a[j], xb[c], x[c]);
        }
    }
}

}  // namespace rows
}  // namespace glass
