// k_blas.cu -- batched BLAS-1/2 and symmetric block-tridiagonal routines
// (Sec. III-B: reductions and BLAS L1-L3; block-tridiagonal matrix-vector
// products and direct solvers of trajectory optimization).
//
//   dot            out[b] = x_b . y_b             thread / warp / block(64)
//   gemv           y = alpha op(A) x + beta y     thread / warp (a row per lane)
//   btd_matvec     y = T x                        warp (a block row per lane)
//   btd_posv       T x = b, T = L L^T blockwise   warp (a block row per lane)
//
// T is symmetric block-tridiagonal: N diagonal blocks D_i (nb x nb) and
// N-1 sub-diagonal blocks O_i = T[i+1][i].  The factorization is the block
// Cholesky recurrence L_0 L_0^T = D_0, W_i = O_i L_i^{-T},
// L_{i+1} L_{i+1}^T = D_{i+1} - W_i W_i^T, computed in place (D_i <- L_i,
// O_i <- W_i), followed by the block forward and backward sweeps.
#include "common.cuh"

namespace glass {
namespace {

template <int T>
__global__ void __launch_bounds__(256) k_dot(int n, const float *x, long long sx, const float *y, long long sy,
                                             float *out, int batch) {
    __shared__ float part[8];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const long long b = (long long)blockIdx.x * (blockDim.x / T) + team;
    if (b >= batch) return;  // whole team
    const float *xb = x + b * sx, *yb = y + b * sy;
    float s = 0.f;
    if (T == 1 && (n & 3) == 0 && ((reinterpret_cast<uintptr_t>(xb) | reinterpret_cast<uintptr_t>(yb)) & 15) == 0) {
        // one problem per thread: 16-byte loads (L1 keeps the rest of each line)
        const float4 *x4 = reinterpret_cast<const float4 *>(xb), *y4 = reinterpret_cast<const float4 *>(yb);
        for (int i = 0; i < (n >> 2); ++i) {
            const float4 a = x4[i], c = y4[i];
            s = fmaf(a.x, c.x, s);
            s = fmaf(a.y, c.y, s);
            s = fmaf(a.z, c.z, s);
            s = fmaf(a.w, c.w, s);
        }
    } else {
        for (int i = rank; i < n; i += T) s = fmaf(xb[i], yb[i], s);
    }
    if constexpr (T > 1) s = warp_sum(s);
    if constexpr (T > 32) {
        const int w = threadIdx.x >> 5;
        if ((rank & 31) == 0) part[w] = s;
        team_sync<T>(1 + team);
        if (rank == 0)
            for (int k = 1; k < T / 32; ++k) s += part[w + k];
    }
    if (rank == 0) out[b] = s;
}

// One problem per thread: y = alpha op(A) x + beta y.
__global__ void __launch_bounds__(256) k_gemv_thread(int trans, int m, int n, float alpha, Mat A, const float *x,
                                                     long long sx, float beta, float *y, long long sy, int batch) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const float *a = A.p + b * A.s, *xb = x + b * sx;
    float *yb = y + b * sy;
    const int rows = trans ? n : m, inner = trans ? m : n;
    for (int i = 0; i < rows; ++i) {
        float s = 0.f;
        for (int l = 0; l < inner; ++l) s = fmaf(trans ? a[(long long)i * A.ld + l] : a[(long long)l * A.ld + i], xb[l], s);
        yb[i] = beta == 0.f ? alpha * s : alpha * s + beta * yb[i];
    }
}

// One problem per warp.  op(A) = A: lane i owns output rows i, i+32
// (coalesced column reads), x broadcast by shuffles; op(A) = A^T: each
// output is a column dot product reduced across the warp.
__global__ void __launch_bounds__(256) k_gemv_warp(int trans, int m, int n, float alpha, Mat A, const float *x,
                                                   long long sx, float beta, float *y, long long sy, int batch) {
    const int lane = threadIdx.x & 31;
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;  // whole warp
    const float *a = A.p + b * A.s, *xb = x + b * sx;
    float *yb = y + b * sy;
    if (!trans) {
        float s0 = 0.f, s1 = 0.f;
        for (int l0 = 0; l0 < n; l0 += 32) {
            const float xv = l0 + lane < n ? xb[l0 + lane] : 0.f;
            const int cnt = min(32, n - l0);
            for (int j = 0; j < cnt; ++j) {
                const float xl = __shfl_sync(GLASS_FULL_MASK, xv, j);
                const float *col = a + (long long)(l0 + j) * A.ld;
                if (lane < m) s0 = fmaf(col[lane], xl, s0);
                if (lane + 32 < m) s1 = fmaf(col[lane + 32], xl, s1);
            }
        }
        if (lane < m) yb[lane] = beta == 0.f ? alpha * s0 : alpha * s0 + beta * yb[lane];
        if (lane + 32 < m) yb[lane + 32] = beta == 0.f ? alpha * s1 : alpha * s1 + beta * yb[lane + 32];
    } else {
        const float x0 = lane < m ? xb[lane] : 0.f, x1 = lane + 32 < m ? xb[lane + 32] : 0.f;
        for (int i = 0; i < n; ++i) {
            const float *col = a + (long long)i * A.ld;
            float s = (lane < m ? col[lane] * x0 : 0.f) + (lane + 32 < m ? col[lane + 32] * x1 : 0.f);
            s = warp_sum(s);
            if (lane == 0) yb[i] = beta == 0.f ? alpha * s : alpha * s + beta * yb[i];
        }
    }
}

// y = T x, one problem per warp, lane r the r-th row of every block row.
template <int NB>
__global__ void __launch_bounds__(256) k_btd_matvec(int nb, int N, const float *D, const float *O, const float *x,
                                                    float *y, int batch) {
    const int r = threadIdx.x & 31;
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;  // whole warp
    const long long bb = (long long)nb * nb;
    const float *Db = D + b * N * bb, *Ob = O + b * (N > 1 ? N - 1 : 0) * bb;
    const float *xb = x + b * N * nb;
    float *yb = y + b * N * nb;
    float xp = 0.f, xc = r < nb ? xb[r] : 0.f;
    for (int i = 0; i < N; ++i) {
        const float xn = (i + 1 < N && r < nb) ? xb[(long long)(i + 1) * nb + r] : 0.f;
        float s = 0.f;
        const float *Di = Db + i * bb;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            if (c < nb) {
                const float xcc = __shfl_sync(GLASS_FULL_MASK, xc, c);
                if (r < nb) s = fmaf(Di[c * nb + r], xcc, s);
                if (i > 0) {
                    const float xpc = __shfl_sync(GLASS_FULL_MASK, xp, c);
                    if (r < nb) s = fmaf(Ob[(i - 1) * bb + c * nb + r], xpc, s);
                }
                if (i + 1 < N) {
                    const float xnc = __shfl_sync(GLASS_FULL_MASK, xn, c);
                    if (r < nb) s = fmaf(Ob[i * bb + r * nb + c], xnc, s);
                }
            }
        }
        if (r < nb) yb[(long long)i * nb + r] = s;
        xp = xc;
        xc = xn;
    }
}

// Block Cholesky solve of T x = b in place (D_i <- L_i lower triangle, O_i
// <- W_i, b <- x), one problem per warp: lane r holds row r of the current
// diagonal block in registers.  Per warp shared memory: L_i and W_i
// row-major with pitch NB+1 (lane-owned rows hit distinct banks), 1/l_jj.
template <int NB>
__global__ void __launch_bounds__(256) k_btd_posv(int nb, int N, float *D, float *O, float *bx, int *info, int batch) {
    constexpr int P = NB + 1;
    extern __shared__ float smem[];
    const int r = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *Ls = smem + w * (2 * NB * P + NB), *Ws = Ls + NB * P, *dinv = Ws + NB * P;
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= batch) return;  // whole warp
    const long long bb = (long long)nb * nb;
    float *Db = D + b * N * bb, *Ob = O + b * (N > 1 ? N - 1 : 0) * bb;
    float *xb = bx + b * N * nb;
    const bool live = r < nb;
    int inf = 0;
    // ------------------------------------------------ factorization
    for (int i = 0; i < N; ++i) {
        float *Di = Db + i * bb;
        float d[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) d[c] = (c < nb && live) ? Di[c * nb + r] : 0.f;
        if (i > 0 && live) {  // D_i - W_{i-1} W_{i-1}^T (row r)
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c < nb) {
                    float s = 0.f;
                    for (int k = 0; k < nb; ++k) s = fmaf(Ws[r * P + k], Ws[c * P + k], s);
                    d[c] -= s;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (j < nb) {
                const float djj = __shfl_sync(GLASS_FULL_MASK, d[j], j);
                if (!(djj > 0.f) && inf == 0) inf = i * nb + j + 1;
                const float l = sqrtf(djj), rl = 1.0f / l;
                if (r == j) d[j] = l;
                else if (r > j) d[j] *= rl;
                if (r == 0) dinv[j] = rl;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    if (k > j && k < nb) {
                        const float lkj = __shfl_sync(GLASS_FULL_MASK, d[j], k);
                        if (r >= k) d[k] = fmaf(-d[j], lkj, d[k]);
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            if (c < nb && live) {
                Ls[r * P + c] = c <= r ? d[c] : 0.f;
                if (c <= r) Di[c * nb + r] = d[c];
            }
        }
        __syncwarp();
        if (i + 1 < N) {  // W_i = O_i L_i^{-T}: row r solves w L_i^T = o
            float *Oi = Ob + i * bb;
            float o[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) o[c] = (c < nb && live) ? Oi[c * nb + r] : 0.f;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j < nb) {
                    float s = o[j];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (k < j) s = fmaf(-o[k], Ls[j * P + k], s);
                    o[j] = s * dinv[j];
                }
            }
            __syncwarp();
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                if (c < nb && live) {
                    Ws[r * P + c] = o[c];
                    Oi[c * nb + r] = o[c];
                }
            }
            __syncwarp();
        }
    }
    if (r == 0) info[b] = inf;
    // ------------------------------------------------ forward: L y = b
    float yp = 0.f;
    for (int i = 0; i < N; ++i) {
        const float *Li = Db + i * bb;
        float t = live ? xb[(long long)i * nb + r] : 0.f;
        if (i > 0) {
            const float *Wp = Ob + (i - 1) * bb;
            for (int c = 0; c < nb; ++c) {
                const float yc = __shfl_sync(GLASS_FULL_MASK, yp, c);
                if (live) t = fmaf(-Wp[c * nb + r], yc, t);
            }
        }
        for (int j = 0; j < nb; ++j) {
            const float yj = __shfl_sync(GLASS_FULL_MASK, t, j) / Li[j * nb + j];
            if (r == j) t = yj;
            else if (r > j && live) t = fmaf(-Li[j * nb + r], yj, t);
        }
        if (live) xb[(long long)i * nb + r] = t;
        yp = t;
    }
    // ------------------------------------------------ backward: L^T x = y
    float xn = 0.f;
    for (int i = N - 1; i >= 0; --i) {
        const float *Li = Db + i * bb;
        float t = live ? xb[(long long)i * nb + r] : 0.f;
        if (i + 1 < N) {
            const float *Wi = Ob + i * bb;
            for (int c = 0; c < nb; ++c) {
                const float xc = __shfl_sync(GLASS_FULL_MASK, xn, c);
                if (live) t = fmaf(-Wi[r * nb + c], xc, t);
            }
        }
        for (int j = nb - 1; j >= 0; --j) {
            const float xj = __shfl_sync(GLASS_FULL_MASK, t, j) / Li[j * nb + j];
            if (r == j) t = xj;
            else if (r < j) t = fmaf(-Li[r * nb + j], xj, t);
        }
        if (live) xb[(long long)i * nb + r] = t;
        xn = t;
    }
}

// ------------------------------------------------ block-Jacobi PCG
// Per-warp shared memory (floats) of k_btd_pcg: the Cholesky factor of one
// diagonal block (pitch NB + 1) and the four vectors x, r, p, w of N*nb
// entries each (element (i, r) of a vector at i * nb + r).
__host__ __device__ inline int pcg_warp_floats(int NB, int nb, int N) { return NB * (NB + 1) + 4 * N * nb; }

// Sum over the lanes of a warp; every lane receives the same bits.
__device__ __forceinline__ float lane_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GLASS_FULL_MASK, v, o);
    return v;
}

// out = T v over the whole problem; returns this lane's share of v'out.
// Lane r forms row r of every block row: D_i v_i + O_{i-1} v_{i-1} +
// O_i^T v_{i+1}, the entries of v read from shared memory as broadcasts.
template <int NB>
__device__ __forceinline__ float pcg_matvec(int nb, int N, const float *Db, const float *Ob, const float *v,
                                            float *out, int r) {
    const long long bb = (long long)nb * nb;
    float dotp = 0.f;
    if (r < nb) {
        for (int i = 0; i < N; ++i) {
            const float *Di = Db + i * bb, *vi = v + i * nb;
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < nb) s = fmaf(Di[c * nb + r], vi[c], s);
            if (i > 0) {
                const float *Op = Ob + (i - 1) * bb, *vp = vi - nb;
#pragma unroll
                for (int c = 0; c < NB; ++c)
                    if (c < nb) s = fmaf(Op[c * nb + r], vp[c], s);
            }
            if (i + 1 < N) {
                const float *On = Ob + i * bb, *vn = vi + nb;
#pragma unroll
                for (int c = 0; c < NB; ++c)
                    if (c < nb) s = fmaf(On[r * nb + c], vn[c], s);
            }
            out[i * nb + r] = s;
            dotp = fmaf(vi[r], s, dotp);
        }
    }
    __syncwarp();
    return dotp;
}

// z = M^{-1} v blockwise with the stored inverses (symmetric, column-major:
// lane r reads row r of each as a coalesced column); returns this lane's
// share of v'z.
template <int NB>
__device__ __forceinline__ float pcg_precond(int nb, int N, const float *Mb, const float *v, float *z, int r) {
    const long long bb = (long long)nb * nb;
    float dotp = 0.f;
    if (r < nb) {
        for (int i = 0; i < N; ++i) {
            const float *Mi = Mb + i * bb, *vi = v + i * nb;
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < nb) s = fmaf(Mi[c * nb + r], vi[c], s);
            z[i * nb + r] = s;
            dotp = fmaf(vi[r], s, dotp);
        }
    }
    __syncwarp();
    return dotp;
}

// Block-Jacobi preconditioned conjugate gradient on the symmetric
// block-tridiagonal T, one problem per warp, lane r the r-th row of every
// block.  Set-up: each D_i is factored in registers (Cholesky, row per
// lane) and D_i^{-1} = L_i^{-T} L_i^{-1} is written to the workspace, lane c
// forming column c by a forward and a backward sweep over L_i in shared
// memory.  Then the textbook recurrence: r = b - T x, z = M^{-1} r, p = z,
// rho = r'z; while k < iters and rho > tol2 * rho0 (and rho > 0): q = T p,
// alpha = rho / p'q (stop if p'q <= 0), x += alpha p, r -= alpha q,
// z = M^{-1} r, p = z + (r'z / rho) p.  The reductions are warp sums, so the
// loop control is uniform over the warp.
template <int NB>
__global__ void __launch_bounds__(256) k_btd_pcg(int nb, int N, const float *D, const float *O, const float *bv,
                                                 float *x, int iters, float tol2, int *done, float *ws, int batch) {
    constexpr int P = NB + 1;
    extern __shared__ float smem[];
    const int r = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = N * nb;
    float *Ls = smem + (long long)w * pcg_warp_floats(NB, nb, N);
    float *xs = Ls + NB * P, *rs = xs + m, *ps = rs + m, *vs = ps + m;
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= batch) return;  // whole warp
    const long long bb = (long long)nb * nb;
    const float *Db = D + b * N * bb, *Ob = O + b * (N > 1 ? N - 1 : 0) * bb;
    float *Mb = ws + b * N * bb;
    const bool live = r < nb;
    // ------------------------------------------ inverses of the diagonal blocks
    for (int i = 0; i < N; ++i) {
        const float *Di = Db + i * bb;
        float d[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) d[c] = (c < nb && live) ? Di[c * nb + r] : 0.f;
        bool fail = false;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (j < nb) {
                const float djj = __shfl_sync(GLASS_FULL_MASK, d[j], j);
                if (!(djj > 0.f)) fail = true;
                const float l = sqrtf(djj), rl = 1.0f / l;
                if (r == j) d[j] = l;
                else if (r > j) d[j] *= rl;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    if (k > j && k < nb) {
                        const float lkj = __shfl_sync(GLASS_FULL_MASK, d[j], k);
                        if (r >= k) d[k] = fmaf(-d[j], lkj, d[k]);
                    }
                }
            }
        }
        if (fail) {  // uniform: every lane saw the same pivots
            if (r == 0) done[b] = -1;
            return;
        }
        if (live)
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < nb) Ls[r * P + c] = c <= r ? d[c] : 0.f;
        __syncwarp();
        if (live) {
            float y[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {  // L y = e_r
                if (j < nb) {
                    float s = j == r ? 1.f : 0.f;
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (k < j) s = fmaf(-Ls[j * P + k], y[k], s);
                    y[j] = s / Ls[j * P + j];
                }
            }
#pragma unroll
            for (int j = NB - 1; j >= 0; --j) {  // L^T z = y
                if (j < nb) {
                    float s = y[j];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (k > j && k < nb) s = fmaf(-Ls[k * P + j], y[k], s);
                    y[j] = s / Ls[j * P + j];
                }
            }
            float *Mi = Mb + i * bb;
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < nb) Mi[r * nb + j] = y[j];  // column r (= row r) of D_i^{-1}
        }
        __syncwarp();
    }
    __threadfence_block();  // the inverses are read back by other lanes of this warp
    __syncwarp();
    // ------------------------------------------ r = b - T x, z = M^{-1} r, p = z
    const float *bb_ = bv + b * m;
    float *xb = x + b * m;
    if (live)
        for (int i = 0; i < N; ++i) xs[i * nb + r] = xb[i * nb + r];
    __syncwarp();
    pcg_matvec<NB>(nb, N, Db, Ob, xs, vs, r);
    if (live)
        for (int i = 0; i < N; ++i) rs[i * nb + r] = bb_[i * nb + r] - vs[i * nb + r];
    __syncwarp();
    float rho = lane_sum(pcg_precond<NB>(nb, N, Mb, rs, ps, r));
    const float rho0 = rho;
    int k = 0;
    while (k < iters && rho > 0.f && rho > tol2 * rho0) {
        const float pq = lane_sum(pcg_matvec<NB>(nb, N, Db, Ob, ps, vs, r));
        if (!(pq > 0.f)) break;
        const float alpha = rho / pq;
        if (live)
            for (int i = 0; i < N; ++i) {
                const int e = i * nb + r;
                xs[e] = fmaf(alpha, ps[e], xs[e]);
                rs[e] = fmaf(-alpha, vs[e], rs[e]);
            }
        __syncwarp();
        const float rho_new = lane_sum(pcg_precond<NB>(nb, N, Mb, rs, vs, r));
        const float beta = rho_new / rho;
        if (live)
            for (int i = 0; i < N; ++i) {
                const int e = i * nb + r;
                ps[e] = fmaf(beta, ps[e], vs[e]);
            }
        __syncwarp();
        rho = rho_new;
        ++k;
    }
    if (live)
        for (int i = 0; i < N; ++i) xb[i * nb + r] = xs[i * nb + r];
    if (r == 0) done[b] = k;
}

int nb_bucket(int nb) { return nb <= 8 ? 8 : nb <= 16 ? 16 : 32; }

}  // namespace

cudaError_t launch_dot(int n, const float *x, long long sx, const float *y, long long sy, float *out, int batch,
                       Placement pl, cudaStream_t st) {
    if (pl.scope == SCOPE_THREAD) {
        const int th = 32 * pl.pack;
        k_dot<1><<<ceil_div(batch, th), th, 0, st>>>(n, x, sx, y, sy, out, batch);
    } else if (pl.scope == SCOPE_WARP) {
        k_dot<32><<<ceil_div(batch, pl.pack), 32 * pl.pack, 0, st>>>(n, x, sx, y, sy, out, batch);
    } else {
        k_dot<64><<<ceil_div(batch, pl.pack), 64 * pl.pack, 0, st>>>(n, x, sx, y, sy, out, batch);
    }
    return cudaPeekAtLastError();
}

cudaError_t launch_gemv(int trans, int m, int n, float alpha, Mat A, const float *x, long long sx, float beta, float *y,
                        long long sy, int batch, Placement pl, cudaStream_t st) {
    if (pl.scope == SCOPE_THREAD) {
        const int th = 32 * pl.pack;
        k_gemv_thread<<<ceil_div(batch, th), th, 0, st>>>(trans, m, n, alpha, A, x, sx, beta, y, sy, batch);
    } else {
        k_gemv_warp<<<ceil_div(batch, pl.pack), 32 * pl.pack, 0, st>>>(trans, m, n, alpha, A, x, sx, beta, y, sy,
                                                                        batch);
    }
    return cudaPeekAtLastError();
}

cudaError_t launch_btd_matvec(int nb, int N, const float *D, const float *O, const float *x, float *y, int batch,
                              int pack, cudaStream_t st) {
    const int grid = ceil_div(batch, pack), th = 32 * pack;
    switch (nb_bucket(nb)) {
        case 8: k_btd_matvec<8><<<grid, th, 0, st>>>(nb, N, D, O, x, y, batch); break;
        case 16: k_btd_matvec<16><<<grid, th, 0, st>>>(nb, N, D, O, x, y, batch); break;
        default: k_btd_matvec<32><<<grid, th, 0, st>>>(nb, N, D, O, x, y, batch); break;
    }
    return cudaPeekAtLastError();
}

cudaError_t launch_btd_posv(int nb, int N, float *D, float *O, float *bx, int *info, int batch, int pack,
                            cudaStream_t st) {
    const int grid = ceil_div(batch, pack), th = 32 * pack;
    const int NB = nb_bucket(nb);
    const size_t sm = (size_t)pack * (2 * NB * (NB + 1) + NB) * 4;
    auto kern = NB == 8 ? k_btd_posv<8> : NB == 16 ? k_btd_posv<16> : k_btd_posv<32>;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(kern), sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, th, sm, st>>>(nb, N, D, O, bx, info, batch);
    return cudaPeekAtLastError();
}

size_t btd_pcg_smem(int nb, int N, int pack) {
    return (size_t)pack * pcg_warp_floats(nb_bucket(nb), nb, N) * 4;
}

cudaError_t launch_btd_pcg(int nb, int N, const float *D, const float *O, const float *b, float *x, int iters,
                           float tol, int *done, float *ws, int batch, int pack, cudaStream_t st) {
    const int grid = ceil_div(batch, pack), th = 32 * pack;
    const int NB = nb_bucket(nb);
    const size_t sm = btd_pcg_smem(nb, N, pack);
    auto kern = NB == 8 ? k_btd_pcg<8> : NB == 16 ? k_btd_pcg<16> : k_btd_pcg<32>;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(kern), sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, th, sm, st>>>(nb, N, D, O, b, x, iters, tol * tol, done, ws, batch);
    return cudaPeekAtLastError();
}

}  // namespace glass
