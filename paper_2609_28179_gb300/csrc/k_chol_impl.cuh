// k_chol_impl.cuh -- batched potrf / potrs / trsm / posv kernels at thread, warp
// and block scope, plus the refinement step of posv (FP64 or compensated
// FP32 residual).
//
// Each kernel wraps a device primitive of dev_chol.cuh with the batched
// load / compute / store of one placement (scope x pack, Sec. III-A).  Thread
// scope stages its 32*pack problems through shared memory with coalesced
// 16-byte streaming loads (column-major input) or reads the interleaved
// layout directly; warp scope loads rows straight into registers (each
// column of a problem is a contiguous, coalesced segment); block scope
// stages each problem into its team's shared memory.  Solves with many
// right-hand sides (trsm at warp and block scope, potrs at block scope)
// give each thread whole columns of X with L broadcast from shared memory.
#pragma once
#include "dev_chol.cuh"
#include "dev_rows.cuh"
#include "dev_chol_tc.cuh"
#include "dev_trsm_tc.cuh"

namespace glass {
namespace {

enum CholOp { C_POTRF = 0, C_POTRS = 1, C_TRSM = 2, C_POSV = 3 };

constexpr bool has_factor(int op) { return op == C_POTRF || op == C_POSV; }
constexpr bool has_rhs(int op) { return op != C_POTRF; }

// ------------------------------------------------------------ thread scope
// Input modes of the thread-scope kernels.  STAGE: the CTA's problems pass
// through shared memory (coalesced 4-byte cp.async, one round trip).
// DIRECT (factorizations): packed column-major batches of order n % 4 == 0
// with 16-byte aligned operands -- each thread reads its own problem's
// columns as 16-byte loads straight from global memory (the lower triangle
// only), no shared memory, so residency is bound by registers alone and
// every load of a thread is in flight at once.
// LAYOUT: the 32-problem interleaved layout, coalesced element by element.
enum ThreadMode { TM_STAGE = 0, TM_DIRECT = 1, TM_LAYOUT = 2 };

template <int OP, int NMAX, bool EXACT, bool REFINE>
__global__ void __launch_bounds__(256) k_chol_thread(int n_rt, int nrhs, Mat A, Mat B, int *info,
                                                     int batch, int num, int mode) {
    extern __shared__ float smem[];
    using TR = Tri<NMAX>;
    const int n = EXACT ? NMAX : n_rt;
    const int G = blockDim.x;
    const int b0 = blockIdx.x * G;
    const int cnt = min(G, batch - b0);
    const int t = threadIdx.x;
    const bool staged = mode == TM_STAGE;
    const bool direct = NMAX % 4 == 0 && mode == TM_DIRECT;
    const int SA = odd_stride(n * n);
    const int SB = has_rhs(OP) ? odd_stride(n * nrhs) : 0;
    float *sa = smem;
    float *sb = smem + G * SA;
    if (staged) {
        stage_in(sa, SA, A, b0, cnt);
        if (has_rhs(OP)) stage_in(sb, SB, B, b0, cnt);
        __syncthreads();
    }
    if (t < cnt) {
        const int b = b0 + t;
        const float *pa = sa + t * SA;
        const float *ga = A.p + (long long)b * A.s;   // DIRECT: packed, ld = n
        float a[TR::size];
        float dinv[NMAX];
        if (direct) {
#pragma unroll
            for (int j = 0; j < NMAX; ++j)
#pragma unroll
                for (int c4 = j / 4; c4 < NMAX / 4; ++c4) {
                    if (j < n && 4 * c4 < n) {
                        const float4 v = __ldcs(reinterpret_cast<const float4 *>(ga + j * n + 4 * c4));
                        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (4 * c4 + u >= j) a[TR::idx(4 * c4 + u, j)] = e[u];
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (4 * c4 + u >= j) a[TR::idx(4 * c4 + u, j)] = 0.f;
                    }
                }
        } else {
#pragma unroll
            for (int j = 0; j < NMAX; ++j)
#pragma unroll
                for (int i = j; i < NMAX; ++i)
                    a[TR::idx(i, j)] = (i < n) ? (staged ? pa[j * n + i] : A.get(b, i, j)) : 0.f;
        }
        if (has_factor(OP)) {
            const int inf = thread::potrf<NMAX, EXACT>(a, dinv, n, (num & NUM_FP64_DIAG) != 0);
            info[b] = inf;
        } else {
#pragma unroll
            for (int j = 0; j < NMAX; ++j) dinv[j] = (j < n) ? 1.0f / a[TR::idx(j, j)] : 0.f;
        }
        if (has_rhs(OP)) {
            float *pb = sb + t * SB;
            float *wb = opaque(pb);
            float *gb = B.p + (long long)b * B.s;      // DIRECT: ldb = n, 16-byte aligned columns
            for (int c = 0; c < nrhs; ++c) {
                float x[NMAX];
                if (direct) {
#pragma unroll
                    for (int c4 = 0; c4 < NMAX / 4; ++c4) {
                        const float4 v = 4 * c4 < n ? __ldcs(reinterpret_cast<const float4 *>(gb + c * n + 4 * c4))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                        x[4 * c4] = v.x;
                        x[4 * c4 + 1] = v.y;
                        x[4 * c4 + 2] = v.z;
                        x[4 * c4 + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < NMAX; ++i)
                        x[i] = (i < n) ? (staged ? pb[c * n + i] : B.get(b, i, c)) : 0.f;
                }
                thread::forward<NMAX, EXACT>(a, dinv, x, n);
                if (OP != C_TRSM) thread::backward_t<NMAX, EXACT>(a, dinv, x, n);
                if (REFINE) {
                    // r = b - A x0 in FP64 or as a compensated FP32 dot
                    // product (A and b are still pristine in the staging
                    // buffers / in global memory).
                    float r[NMAX];
                    const bool dot2 = (num & NUM_DOT2_RESIDUAL) != 0;
#pragma unroll
                    for (int i = 0; i < NMAX; ++i) {
                        if (i < n) {
                            const float bi = staged ? pb[c * n + i] : B.get(b, i, c);
                            auto aik = [&](int k) {
                                return (k <= i) ? (staged ? pa[k * n + i] : A.get(b, i, k))
                                                : (staged ? pa[i * n + k] : A.get(b, k, i));
                            };
                            if (dot2) {
                                Dot2 d;
                                d.init(bi);
#pragma unroll
                                for (int k = 0; k < NMAX; ++k)
                                    if (k < n) d.sub(aik(k), x[k]);
                                r[i] = d.value();
                            } else {
                                double acc = (double)bi;
#pragma unroll
                                for (int k = 0; k < NMAX; ++k)
                                    if (k < n) acc = fma(-(double)aik(k), (double)x[k], acc);
                                r[i] = (float)acc;
                            }
                        } else {
                            r[i] = 0.f;
                        }
                    }
                    thread::forward<NMAX, EXACT>(a, dinv, r, n);
                    thread::backward_t<NMAX, EXACT>(a, dinv, r, n);
#pragma unroll
                    for (int i = 0; i < NMAX; ++i) x[i] += r[i];
                }
                if (direct) {
                    float *wg = opaque(gb);
#pragma unroll
                    for (int c4 = 0; c4 < NMAX / 4; ++c4)
                        if (4 * c4 < n)
                            __stcs(reinterpret_cast<float4 *>(wg + c * n + 4 * c4),
                                   make_float4(x[4 * c4], x[4 * c4 + 1], x[4 * c4 + 2], x[4 * c4 + 3]));
                } else {
#pragma unroll
                    for (int i = 0; i < NMAX; ++i)
                        if (i < n) {
                            if (staged) wb[c * n + i] = x[i];
                            else B.set(b, i, c, x[i]);
                        }
                }
            }
        }
        if (has_factor(OP)) {
            if (direct) {
                // whole 16-byte groups below the diagonal; the group that
                // holds the diagonal element by element (the strict upper
                // triangle keeps its contents)
                float *wg = opaque(A.p + (long long)b * A.s);
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
#pragma unroll
                    for (int c4 = j / 4; c4 < NMAX / 4; ++c4) {
                        if (j < n && 4 * c4 < n) {
                            if (4 * c4 >= j) {
                                __stcs(reinterpret_cast<float4 *>(wg + j * n + 4 * c4),
                                       make_float4(a[TR::idx(4 * c4, j)], a[TR::idx(4 * c4 + 1, j)],
                                                   a[TR::idx(4 * c4 + 2, j)], a[TR::idx(4 * c4 + 3, j)]));
                            } else {
#pragma unroll
                                for (int u = 0; u < 4; ++u)
                                    if (4 * c4 + u >= j) wg[j * n + 4 * c4 + u] = a[TR::idx(4 * c4 + u, j)];
                            }
                        }
                    }
            } else {
                float *wa = opaque(sa + t * SA);
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
#pragma unroll
                    for (int i = j; i < NMAX; ++i)
                        if (i < n) {
                            if (staged) wa[j * n + i] = a[TR::idx(i, j)];
                            else A.set(b, i, j, a[TR::idx(i, j)]);
                        }
            }
        }
    }
    if (staged) {
        __syncthreads();
        if (has_factor(OP)) stage_out(sa, SA, A, b0, cnt);
        if (has_rhs(OP)) stage_out(sb, SB, B, b0, cnt);
    }
}

// -------------------------------------------------------------- warp scope
// Row-distributed Cholesky / solve: lane i holds row i (and i+32).  The
// refinement step is a separate instantiation (REFINE) so the plain kernel
// does not carry its registers.  Dynamic shared memory: one NMAX-float
// column buffer per warp.
template <int OP, int NMAX, bool REFINE>
__global__ void __launch_bounds__(256, NMAX <= 16 ? 3 : (NMAX == 32 ? 2 : 1)) k_chol_warp(int n, int nrhs, Mat A, Mat B, int *info, int batch,
                                                   int num) {
    constexpr int R = warp::Rows<NMAX>::R;
    constexpr int AP = NMAX + 1;  // odd pitch of the refinement copy of A
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31;
    float *col = smem + (threadIdx.x >> 5) * (NMAX + (REFINE ? NMAX * AP : 0));
    float *As = col + NMAX;  // REFINE only: original A, element (i,k) at k*AP + i
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;  // whole warp
    float a[R][NMAX];
    float rd[R];
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            a[q][k] = (k < n && i < n && k <= i) ? A.cget(b, i, k) : 0.f;
            if (REFINE && k < n && i < n && k <= i) As[k * AP + i] = a[q][k];
        }
    if (has_factor(OP)) {
        const int inf = warp::potrf<NMAX>(a, rd, n, (num & NUM_FP64_DIAG) != 0, col);
        if (lane == 0) info[b] = inf;
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            float dii = 1.f;
#pragma unroll
            for (int k = 0; k < NMAX; ++k)
                if (k == i) dii = a[q][k];
            rd[q] = (i < n) ? 1.0f / dii : 0.f;
        }
    }
    if (has_rhs(OP)) {
        for (int c = 0; c < nrhs; ++c) {
            float x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                x[q] = (i < n) ? B.cget(b, i, c) : 0.f;
            }
            warp::forward<NMAX>(a, rd, x, n);
            if (OP != C_TRSM) warp::backward_t<NMAX>(a, rd, x, n);
            if (REFINE) {
                // r_i = b_i - sum_k a_ik x_k from the original A kept in
                // shared memory (lower triangle, odd pitch: conflict free):
                // in FP64 with four independent partial sums per row (they
                // hide the FP64 latency), or as two compensated FP32 sums.
                float r[R];
                auto xk_of = [&](int k) {
                    float xk = 0.f;
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const float v = __shfl_sync(GLASS_FULL_MASK, x[q], k & 31);
                        if ((k >> 5) == q) xk = v;
                    }
                    return xk;
                };
                if ((num & NUM_DOT2_RESIDUAL) != 0) {
                    Dot2 d[R][2];
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int i = lane + 32 * q;
                        d[q][0].init((i < n) ? B.cget(b, i, c) : 0.f);
                        d[q][1].init(0.f);
                    }
#pragma unroll 4
                    for (int k = 0; k < NMAX; ++k) {
                        if (k < n) {
                            const float xk = xk_of(k);
#pragma unroll
                            for (int q = 0; q < R; ++q) {
                                const int i = lane + 32 * q;
                                if (i < n) d[q][k & 1].sub((k <= i) ? As[k * AP + i] : As[i * AP + k], xk);
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        d[q][0].merge(d[q][1]);
                        r[q] = d[q][0].value();
                    }
                } else {
                    double acc[R][4];
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int i = lane + 32 * q;
                        acc[q][0] = (i < n) ? (double)B.cget(b, i, c) : 0.0;
                        acc[q][1] = acc[q][2] = acc[q][3] = 0.0;
                    }
#pragma unroll 4
                    for (int k = 0; k < NMAX; ++k) {
                        if (k < n) {
                            const float xk = xk_of(k);
#pragma unroll
                            for (int q = 0; q < R; ++q) {
                                const int i = lane + 32 * q;
                                if (i < n) {
                                    const float aik = (k <= i) ? As[k * AP + i] : As[i * AP + k];
                                    acc[q][k & 3] = fma(-(double)aik, (double)xk, acc[q][k & 3]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < R; ++q) r[q] = (float)((acc[q][0] + acc[q][1]) + (acc[q][2] + acc[q][3]));
                }
                warp::forward<NMAX>(a, rd, r, n);
                warp::backward_t<NMAX>(a, rd, r, n);
#pragma unroll
                for (int q = 0; q < R; ++q) x[q] += r[q];
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (i < n) B.cset(b, i, c, x[q]);
            }
        }
    }
    if (has_factor(OP)) {
        float *wa = opaque(A.p + (long long)b * A.s);
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (k < n && i < n && k <= i) wa[(long long)k * A.ld + i] = a[q][k];
            }
    }
}

// Per-warp shared memory (floats) of k_chol_tc: A, 1/l_jj and two 16-float
// broadcast segments.  The refinement step keeps the first solution in the
// padding rows NMAX..NMAX+7 of A's first columns (rows no kernel step
// touches), so refinement costs no shared memory and no resident warps.
template <int NMAX>
constexpr int tc_floats() {
    return NMAX * tcwarp::Shape<NMAX>::LD + NMAX + 32;
}

// x_k of the refinement in A's padding: as a double (four per column) for
// the FP64 residual, as a float (eight per column) for the compensated one.
template <int NMAX>
__device__ __forceinline__ double *xpad_d(float *As, int k) {
    return reinterpret_cast<double *>(As + (k >> 2) * tcwarp::Shape<NMAX>::LD + NMAX) + (k & 3);
}
template <int NMAX>
__device__ __forceinline__ float *xpad_f(float *As, int k) {
    return As + (k >> 3) * tcwarp::Shape<NMAX>::LD + NMAX + (k & 7);
}

// The entries a_ik of the ORIGINAL symmetric operand in global memory (lower
// triangle, still intact: the factor is written back last) for the lane's
// rows i = lane + 32 q and the CW columns k0..k0+CW-1, all loads issued before
// any is used (the residual waits on these loads, not on its arithmetic):
// below the diagonal from column k (coalesced over the lanes), above it as
// a_ki from the row's own column; zero outside the order.
template <int R, int CW>
__device__ __forceinline__ void residual_chunk(const float *ga, long long lda, int n, int k0, float (&av)[R][CW]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int kk = 0; kk < CW; ++kk)
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q, k = k0 + kk;
            av[q][kk] = (i < n && k < n) ? (i >= k ? ga[(long long)k * lda + i] : ga[(long long)i * lda + k]) : 0.f;
        }
}

// Runs use(av, k0) over the column chunks of the residual (CW = kResCW<NMAX>
// columns).  The 64-row kernel keeps the loads of the next 8-column chunk in
// flight while a chunk is used (two register buffers; refined posv n = 64
// at batch 16384: 536 -> 519 us with the FP64 residual, 445 -> 425 us with
// the compensated one); the 32-row kernel loads 16 columns at a time into
// one buffer (the second buffer cost it resident warps: 113 -> 131 us).
// k0 < n <= NMAX, so every chunk used lies inside the operand's columns,
// and a chunk past n is never loaded.
template <int NMAX>
constexpr int kResCW = NMAX == 64 ? 8 : 16;
template <int NMAX, typename Use>
__device__ __forceinline__ void residual_pipeline(const float *ga, long long lda, int n, Use use) {
    constexpr int R = tcwarp::Shape<NMAX>::R, CW = kResCW<NMAX>;
    float a0[R][CW];
    if constexpr (NMAX == 64) {
        float a1[R][CW];
        residual_chunk<R, CW>(ga, lda, n, 0, a0);
        for (int k0 = 0; k0 < n; k0 += 2 * CW) {
            const bool second = k0 + CW < n;
            if (second) residual_chunk<R, CW>(ga, lda, n, k0 + CW, a1);
            use(a0, k0);
            if (second) {
                if (k0 + 2 * CW < n) residual_chunk<R, CW>(ga, lda, n, k0 + 2 * CW, a0);
                use(a1, k0 + CW);
            }
        }
    } else {
        for (int k0 = 0; k0 < n; k0 += CW) {
            residual_chunk<R, CW>(ga, lda, n, k0, a0);
            use(a0, k0);
        }
    }
}

// r = b - A x in FP64 for one right-hand side of the tensor-core posv (lane
// rows i = lane + 32 q, x_k from A's padding as FP64): n fused multiply-adds
// per row in two partial sums, and, in the 64-row kernel, the widening of
// A's entries on the FP64 pipe (the 32-row kernel widens them on the
// integer pipe, f2d_bits).
template <int NMAX>
__device__ __forceinline__ void residual_f64(const float *ga, long long lda, float *As,
                                             const float (&bq)[tcwarp::Shape<NMAX>::R], int n,
                                             float (&r)[tcwarp::Shape<NMAX>::R]) {
    constexpr int R = tcwarp::Shape<NMAX>::R;
    double acc[R][2];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        acc[q][0] = (double)bq[q];
        acc[q][1] = 0.0;
    }
    // Widening on the integer pipe measured faster for the 32-row kernel
    // (refined solve at batch 16384: 128 vs 155 us) and slower for the
    // 64-row one (731 vs 605 us), which keeps the hardware conversion.
    auto widen = [](float a) { return NMAX == 32 ? f2d_bits(a) : (double)a; };
    residual_pipeline<NMAX>(ga, lda, n, [&](const float (&av)[R][kResCW<NMAX>], int k0) {
#pragma unroll
        for (int kk = 0; kk < kResCW<NMAX>; ++kk) {
            const double xk = *xpad_d<NMAX>(As, k0 + kk);  // zero beyond n
#pragma unroll
            for (int q = 0; q < R; ++q) acc[q][kk & 1] = fma(-widen(av[q][kk]), xk, acc[q][kk & 1]);
        }
    });
#pragma unroll
    for (int q = 0; q < R; ++q) r[q] = (float)(acc[q][0] + acc[q][1]);
}

// The same residual as a compensated FP32 dot product (Dot2), x_k from A's
// padding as FP32, two partial sums per row merged at the end: about ten
// FP32 operations per term on the wide FP32 pipe instead of a widening and
// a fused multiply-add on the FP64 one.
template <int NMAX>
__device__ __forceinline__ void residual_dot2(const float *ga, long long lda, float *As,
                                              const float (&bq)[tcwarp::Shape<NMAX>::R], int n,
                                              float (&r)[tcwarp::Shape<NMAX>::R]) {
    constexpr int R = tcwarp::Shape<NMAX>::R;
    Dot2 d[R][2];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        d[q][0].init(bq[q]);
        d[q][1].init(0.f);
    }
    residual_pipeline<NMAX>(ga, lda, n, [&](const float (&av)[R][kResCW<NMAX>], int k0) {
#pragma unroll
        for (int kk = 0; kk < kResCW<NMAX>; ++kk) {
            const float xk = *xpad_f<NMAX>(As, k0 + kk);  // zero beyond n
#pragma unroll
            for (int q = 0; q < R; ++q) d[q][kk & 1].sub(av[q][kk], xk);
        }
    });
#pragma unroll
    for (int q = 0; q < R; ++q) {
        d[q][0].merge(d[q][1]);
        r[q] = d[q][0].value();
    }
}

// Warp scope, orders 17..64: blocked Cholesky with tensor-core trailing
// updates (dev_chol_tc.cuh) on the problem held in the warp's shared memory;
// the solves run against L in shared memory.  RF: one refinement step per
// right-hand side -- r = b - A x0 in FP64 (or as a compensated FP32 dot
// product) from the original A (still intact in global memory: the factor
// is written back last), dx = A^{-1} r with
// the factor, x1 = x0 + dx.  (A shared-memory copy of A halves the resident
// warps and measured slower.)
// Orders 17..32 without refinement cap the registers at 64, so 32 warps fit
// on an SM instead of 28 (posv n = 32 at batch 16384: 60 -> 58 us).
template <int OP, int NMAX, bool RF>
__global__ void __launch_bounds__(256, NMAX == 32 && !RF ? 4 : 1) k_chol_tc(int n, int nrhs, Mat A, Mat B, int *info, int batch, int num) {
    constexpr int LD = tcwarp::Shape<NMAX>::LD;
    constexpr int R = tcwarp::Shape<NMAX>::R;
    extern __shared__ __align__(16) float smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *As = smem + w * tc_floats<NMAX>();
    float *dv = As + NMAX * LD;
    float *bc = dv + NMAX;
    const int b = blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= batch) return;  // whole warp
    tcwarp::stage_async<NMAX, true>(As, A.p + (long long)b * A.s, A.ld, n);
    tcwarp::wait_first();  // the first panel starts while columns 16.. arrive
    const int inf = tcwarp::potrf<NMAX>(As, n, dv, bc, (num & NUM_FP64_DIAG) != 0);
    if (lane == 0) info[b] = inf;
    if (has_rhs(OP)) {
        for (int c = 0; c < nrhs; ++c) {
            float x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                x[q] = (i < n) ? B.cget(b, i, c) : 0.f;
            }
            float bq[R];
#pragma unroll
            for (int q = 0; q < R; ++q) bq[q] = x[q];
            tcwarp::potrs<NMAX>(As, dv, x, n);
            if constexpr (RF) {
                float r[R];
                if ((num & NUM_DOT2_RESIDUAL) != 0) {
#pragma unroll
                    for (int q = 0; q < R; ++q) *xpad_f<NMAX>(As, lane + 32 * q) = x[q];  // rows >= n hold 0
                    __syncwarp();
                    residual_dot2<NMAX>(A.p + (long long)b * A.s, A.ld, As, bq, n, r);
                } else {
#pragma unroll
                    for (int q = 0; q < R; ++q) *xpad_d<NMAX>(As, lane + 32 * q) = (double)x[q];
                    __syncwarp();
                    residual_f64<NMAX>(A.p + (long long)b * A.s, A.ld, As, bq, n, r);
                }
                __syncwarp();  // x is rewritten for the next right-hand side
                tcwarp::potrs<NMAX>(As, dv, r, n);
#pragma unroll
                for (int q = 0; q < R; ++q) x[q] += r[q];
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = lane + 32 * q;
                if (i < n) B.cset(b, i, c, x[q]);
            }
        }
    }
    tcwarp::unstage<NMAX, true>(A.p + (long long)b * A.s, A.ld, As, n);
}

// Solves with many right-hand sides, orders 33..64 (trsm; potrs when BOTH):
// a team of T threads per problem, blocked with tensor-core updates
// (dev_trsm_tc.cuh); each warp of the team takes chunks of 32 right-hand
// sides.
template <int T, bool BOTH>
__global__ void __launch_bounds__(256, 1) k_solve_tc(int n, int nrhs, Mat L, Mat B, int batch) {
    using namespace tctrsm;
    constexpr int W = T / 32;
    extern __shared__ __align__(16) float smem[];
    const int team = threadIdx.x / T, rank = threadIdx.x % T, w = rank >> 5;
    const int b = blockIdx.x * (blockDim.x / T) + team;
    const int bar = 1 + team;
    float *Ls = smem + team * floats<T>();
    float *dv = Ls + NMAX * LD;
    float *Bs = dv + NMAX + w * CW * LDB;
    if (b >= batch || nrhs <= 0) return;  // whole team
    const float *gl = L.p + (long long)b * L.s;
    float *gb = B.p + (long long)b * B.s;
    const bool vec = (n & 3) == 0 && (L.ld & 3) == 0 && (B.ld & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(gl) | reinterpret_cast<uintptr_t>(gb)) & 15) == 0;
    stage_cols<true>(Ls, LD, gl, L.ld, n, n, NMAX, vec, rank, T);
    int c0 = w * CW;
    if (c0 < nrhs)
        stage_cols<false>(Bs, LDB, gb + (long long)c0 * B.ld, B.ld, n, min(CW, nrhs - c0), CW, vec, rank & 31, 32);
    cp_async_wait_all();
    team_sync<T>(bar);
    for (int i = rank; i < NMAX; i += T) dv[i] = i < n ? 1.0f / Ls[i * LD + i] : 0.f;
    team_sync<T>(bar);
    for (bool first = true; c0 < nrhs; c0 += W * CW, first = false) {
        const int cols = min(CW, nrhs - c0);
        if (!first) {
            stage_cols<false>(Bs, LDB, gb + (long long)c0 * B.ld, B.ld, n, cols, CW, vec, rank & 31, 32);
            cp_async_wait_all();
            __syncwarp();
        }
        forward(Ls, dv, Bs, n);
        if (BOTH) backward_t(Ls, dv, Bs, n);
        store_cols(gb + (long long)c0 * B.ld, B.ld, Bs, n, cols, vec);
        __syncwarp();
    }
}

// Solves with many right-hand sides (trsm; potrs when BOTH): a team of T
// threads per problem, L (lower triangle) and B staged in shared memory,
// each thread solving whole columns of X in registers with L read as
// 16-byte broadcasts.  Packed, 16-byte aligned operands of order n % 4 == 0
// are staged with cp.async 16-byte copies (only the chunks of L that hold
// lower-triangle entries); anything else with plain loads.  Per problem in
// shared memory: L (NMAX x NMAX), 1/l_ii, B (pitch col_pitch(n)).
template <int NMAX, int T, bool BOTH>
__global__ void __launch_bounds__(256, 1) k_solve_cols(int n, int nrhs, Mat L, Mat B, int batch) {
    extern __shared__ __align__(16) float smem[];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const int P = blockDim.x / T;
    const int b = blockIdx.x * P + team;
    const int bar = 1 + team;
    const int ldb = col_pitch(n);
    const int per = NMAX * NMAX + NMAX + nrhs * ldb;
    float *Ls = smem + team * per;
    float *dv = Ls + NMAX * NMAX;
    float *Bs = dv + NMAX;
    if (b >= batch) return;
    const float *gl = L.p + (long long)b * L.s;
    const float *gb = B.p + (long long)b * B.s;
    const bool vec = (n & 3) == 0 && L.ld == n && B.ld == n &&
                     ((reinterpret_cast<uintptr_t>(gl) | reinterpret_cast<uintptr_t>(gb)) & 15) == 0;
    if (vec) {
        const int q4 = n >> 2;  // 16-byte chunks per column
        for (int e = rank; e < n * q4; e += T) {
            const int j = e / q4, q = e - j * q4;
            if (4 * q + 3 >= j) cp_async16(Ls + j * NMAX + 4 * q, gl + j * n + 4 * q);
        }
        for (int e = rank; e < nrhs * q4; e += T) {
            const int c = e / q4, q = e - c * q4;
            cp_async16(Bs + c * ldb + 4 * q, gb + c * n + 4 * q);
        }
        cp_async_wait_all();
    } else {
        for (int e = rank; e < n * n; e += T) {
            const int j = e / n, i = e - j * n;
            if (i >= j) Ls[j * NMAX + i] = L.cget(b, i, j);
        }
        for (int e = rank; e < n * nrhs; e += T) {
            const int c = e / n, i = e - c * n;
            Bs[c * ldb + i] = B.cget(b, i, c);
        }
    }
    team_sync<T>(bar);
    for (int i = rank; i < n; i += T) dv[i] = 1.0f / Ls[i * NMAX + i];
    team_sync<T>(bar);
    for (int c = rank; c < nrhs; c += T) {
        // the column is read and written as 16-byte vectors: with the
        // col_pitch stride, 8 consecutive threads touch 8 distinct bank groups
        float x[NMAX];
        const float4 *xc4 = reinterpret_cast<const float4 *>(Bs + c * ldb);
#pragma unroll
        for (int i4 = 0; i4 < NMAX / 4; ++i4) {
            const float4 v = 4 * i4 < n ? xc4[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[4 * i4] = v.x; x[4 * i4 + 1] = v.y; x[4 * i4 + 2] = v.z; x[4 * i4 + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < NMAX; ++i)
            if (i >= n) x[i] = 0.f;
        warp::forward_cols<NMAX>(Ls, dv, x, n);
        if (BOTH) warp::backward_t_cols<NMAX>(Ls, dv, x, n);
        float4 *wc4 = reinterpret_cast<float4 *>(opaque(Bs + c * ldb));
#pragma unroll
        for (int i4 = 0; i4 < NMAX / 4; ++i4)
            if (4 * i4 < n) wc4[i4] = make_float4(x[4 * i4], x[4 * i4 + 1], x[4 * i4 + 2], x[4 * i4 + 3]);
    }
    team_sync<T>(bar);
    float *wg = B.p + (long long)b * B.s;
    if (vec) {
        const int q4 = n >> 2;
        for (int e = rank; e < nrhs * q4; e += T) {
            const int c = e / q4, q = e - c * q4;
            __stcs(reinterpret_cast<float4 *>(wg + c * n + 4 * q), *reinterpret_cast<const float4 *>(Bs + c * ldb + 4 * q));
        }
    } else {
        for (int e = rank; e < n * nrhs; e += T) {
            const int c = e / n, i = e - c * n;
            B.cset(b, i, c, Bs[c * ldb + i]);
        }
    }
}

// ------------------------------------------------------------- block scope
// Row team (dev_rows.cuh): 64 threads per problem, thread i owns row i,
// right-hand sides handled RS = 4 at a time.  The refinement residual
// r = b - A x0 is formed in FP64 (or as a compensated FP32 dot product) from
// A re-read in global memory (L is written back last) and the solved x
// broadcast through shared memory.
constexpr int kRSmax = 4;

template <int NMAX>
constexpr int rows_team_floats() {
    return ((rows::Scratch<NMAX, kRSmax>::floats + NMAX * kRSmax + 3) / 4) * 4;
}

template <int OP, int NMAX, bool REFINE, int kRS>
__global__ void __launch_bounds__(256, 1) k_chol_rows(int n, int nrhs, Mat A, Mat B, int *info, int batch,
                                                   int num) {
    extern __shared__ __align__(16) float smem[];
    const int team = threadIdx.x / rows::T, i = threadIdx.x % rows::T;
    const int b = blockIdx.x * (blockDim.x / rows::T) + team;
    const int bid = 1 + team;
    float *base = smem + team * rows_team_floats<NMAX>();
    rows::Scratch<NMAX, kRS> s(base);
    float *xall = base + rows::Scratch<NMAX, kRSmax>::floats;  // [NMAX][kRS]
    if (b >= batch) return;  // the whole team leaves together
    float a[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) a[k] = (k < n && i < n && k <= i) ? A.cget(b, i, k) : 0.f;
    const int inf = rows::potrf<NMAX, kRS>(a, n, i, (num & NUM_FP64_DIAG) != 0, s, bid);
    if (i == 0) info[b] = inf;
    if (has_rhs(OP)) {
        for (int c0 = 0; c0 < nrhs; c0 += kRS) {
            float x[kRS];
#pragma unroll
            for (int c = 0; c < kRS; ++c) x[c] = (i < n && c0 + c < nrhs) ? B.cget(b, i, c0 + c) : 0.f;
            rows::forward<NMAX, kRS>(a, x, n, i, s, bid);
            rows::backward_t<NMAX, kRS>(a, x, n, i, s, bid);
            if (REFINE) {
                if (i < n)
#pragma unroll
                    for (int c = 0; c < kRS; ++c) xall[i * kRS + c] = x[c];
                rows::bar(bid);
                float r[kRS];
                const bool dot2 = (num & NUM_DOT2_RESIDUAL) != 0;
#pragma unroll
                for (int c = 0; c < kRS; ++c) {
                    const float bi = (i < n && c0 + c < nrhs) ? B.cget(b, i, c0 + c) : 0.f;
                    if (dot2) {
                        Dot2 d;
                        d.init(bi);
                        if (i < n)
                            for (int k = 0; k < n; ++k)
                                d.sub((k <= i) ? A.cget(b, i, k) : A.cget(b, k, i), xall[k * kRS + c]);
                        r[c] = d.value();
                    } else {
                        double acc = (double)bi;
                        if (i < n)
                            for (int k = 0; k < n; ++k) {
                                const float aik = (k <= i) ? A.cget(b, i, k) : A.cget(b, k, i);
                                acc = fma(-(double)aik, (double)xall[k * kRS + c], acc);
                            }
                        r[c] = (float)acc;
                    }
                }
                rows::forward<NMAX, kRS>(a, r, n, i, s, bid);
                rows::backward_t<NMAX, kRS>(a, r, n, i, s, bid);
#pragma unroll
                for (int c = 0; c < kRS; ++c) x[c] += r[c];
                rows::bar(bid);  // xall reads done before a later pass rewrites it
            }
            if (i < n) {
                float *wb = opaque(B.p + (long long)b * B.s);
#pragma unroll
                for (int c = 0; c < kRS; ++c)
                    if (c0 + c < nrhs) wb[(long long)(c0 + c) * B.ld + i] = x[c];
            }
        }
    }
    float *wa = opaque(A.p + (long long)b * A.s);
#pragma unroll
    for (int k = 0; k < NMAX; ++k)
        if (k < n && i < n && k <= i) wa[(long long)k * A.ld + i] = a[k];
}

// ---------------------------------------------------------------- dispatch
template <typename K, typename... Args>
cudaError_t launch_k(K kern, int grid, int threads, size_t smem, cudaStream_t st, Args... args) {
    {
        cudaError_t e = prepare(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, threads, smem, st>>>(args...);
    return cudaPeekAtLastError();
}

constexpr size_t kMaxSmem = 227 * 1024;

inline int nmax_bucket(int n) { return n <= 8 ? 8 : n <= 16 ? 16 : n <= 32 ? 32 : 64; }

// Thread-scope instantiations: exact orders of the placement sweep and
// buckets (runtime order <= NMAX) for the rest.
template <int OP, bool RF>
cudaError_t thread_dispatch(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, int pack,
                            int num, cudaStream_t st) {
    const int G = 32 * pack;
    const bool aligned = ((reinterpret_cast<uintptr_t>(A.p) | (has_rhs(OP) ? reinterpret_cast<uintptr_t>(B.p) : 0)) &
                          15) == 0;
    // DIRECT for the factoring operations (posv n = 12 at batch 16384: 8.9 us
    // against 12.9 staged); the triangular solves with n right-hand sides
    // measured slower that way (trsm n = 12: 17.2 against 14.6 us) and stage
    const int mode = A.layout != GLASS_LAYOUT_COLMAJOR ? TM_LAYOUT
                     : (has_factor(OP) && (n & 3) == 0 && aligned && A.packed() && (!has_rhs(OP) || B.ld == n) &&
                        (!has_rhs(OP) || (B.s & 3) == 0) && !RF)
                         ? TM_DIRECT
                         : TM_STAGE;
    const size_t smem =
        mode == TM_STAGE ? (size_t)G * (odd_stride(n * n) + (has_rhs(OP) ? odd_stride(n * nrhs) : 0)) * 4 : 0;
    const int grid = ceil_div(batch, G);
#define GL_T(N, EX) \
    launch_k(k_chol_thread<OP, N, EX, RF>, grid, G, smem, st, n, nrhs, A, B, info, batch, num, mode)
    switch (n) {
        case 3: return GL_T(3, true);
        case 6: return GL_T(6, true);
        case 7: return GL_T(7, true);
        case 12: return GL_T(12, true);
        case 14: return GL_T(14, true);
        default: break;
    }
    if (n <= 2) return GL_T(2, false);
    if (n <= 4) return GL_T(4, false);
    if (n <= 8) return GL_T(8, false);
    if (n <= 12) return GL_T(12, false);
    return GL_T(16, false);
#undef GL_T
}

// Shared memory of the blocked tensor-core Cholesky, per warp (bytes).
inline size_t tc_smem(int n) {  // the refinement step lives in A's padding: no extra
    return (size_t)(n > 32 ? tc_floats<64>() : tc_floats<32>()) * 4;
}

// Shared memory of the many-right-hand-side solve kernels, per problem
// (bytes), for a team of T threads: column-per-thread up to order 32,
// blocked tensor-core form above.
// Order bucket of the column solve: an exact 24 besides the powers of two
// (trsm n = 24 at batch 16384 ran padded to 32 rows).
inline int cols_bucket(int n) { return n <= 8 ? 8 : n <= 16 ? 16 : n <= 24 ? 24 : n <= 32 ? 32 : 64; }

inline size_t solve_cols_per(int n, int nrhs, int T) {
    if (n > 32) return (size_t)(T == 32 ? tctrsm::floats<32>() : tctrsm::floats<64>()) * 4;
    const int N = cols_bucket(n);
    return (size_t)(N * N + N + (size_t)nrhs * col_pitch(n)) * 4;
}

template <int NMAX, int T, bool BOTH>
cudaError_t launch_solve_cols(int n, int nrhs, const Mat &L, const Mat &B, int batch, int pack, cudaStream_t st) {
    auto kern = k_solve_cols<NMAX, T, BOTH>;
    const size_t sm = solve_cols_per(n, nrhs, T) * pack;
    cudaError_t e = prepare(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<ceil_div(batch, pack), T * pack, sm, st>>>(n, nrhs, L, B, batch);
    return cudaPeekAtLastError();
}

template <int T, bool BOTH>
cudaError_t solve_cols_dispatch(int n, int nrhs, const Mat &L, const Mat &B, int batch, int pack, cudaStream_t st) {
    if (n > 32) {
        auto kern = k_solve_tc<T, BOTH>;
        const size_t sm = (size_t)tctrsm::floats<T>() * 4 * pack;
        cudaError_t e = prepare(kern, sm);
        if (e != cudaSuccess) return e;
        kern<<<ceil_div(batch, pack), T * pack, sm, st>>>(n, nrhs, L, B, batch);
        return cudaPeekAtLastError();
    }
    switch (cols_bucket(n)) {
        case 8: return launch_solve_cols<8, T, BOTH>(n, nrhs, L, B, batch, pack, st);
        case 16: return launch_solve_cols<16, T, BOTH>(n, nrhs, L, B, batch, pack, st);
        case 24: return launch_solve_cols<24, T, BOTH>(n, nrhs, L, B, batch, pack, st);
        case 32: return launch_solve_cols<32, T, BOTH>(n, nrhs, L, B, batch, pack, st);
        default: return launch_solve_cols<64, T, BOTH>(n, nrhs, L, B, batch, pack, st);
    }
}

template <int OP, bool RF>
cudaError_t warp_dispatch(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, int pack,
                          int num, cudaStream_t st) {
    if constexpr (OP == C_TRSM) {
        return solve_cols_dispatch<32, false>(n, nrhs, A, B, batch, pack, st);
    } else {
        if constexpr (has_factor(OP)) {
            if (n > 16) {
                const int grid = ceil_div(batch, pack);
                if (n > 32)
                    return launch_k(k_chol_tc<OP, 64, RF>, grid, 32 * pack, tc_smem(n) * pack, st, n, nrhs, A, B,
                                    info, batch, num);
                return launch_k(k_chol_tc<OP, 32, RF>, grid, 32 * pack, tc_smem(n) * pack, st, n, nrhs, A, B, info,
                                batch, num);
            }
        }
        const int threads = 32 * pack;
        const int grid = ceil_div(batch, pack);
        const int N = nmax_bucket(n);
        const size_t sm = (size_t)pack * (N + (RF ? N * (N + 1) : 0)) * 4;
#define GL_W(NN) launch_k(k_chol_warp<OP, NN, RF>, grid, threads, sm, st, n, nrhs, A, B, info, batch, num)
        switch (N) {
            case 8: return GL_W(8);
            case 16: return GL_W(16);
            case 32: return GL_W(32);
            default: return GL_W(64);
        }
#undef GL_W
    }
}

inline size_t rows_team_bytes(int n) {
    switch (nmax_bucket(n)) {
        case 8: return rows_team_floats<8>() * 4;
        case 16: return rows_team_floats<16>() * 4;
        case 32: return rows_team_floats<32>() * 4;
        default: return rows_team_floats<64>() * 4;
    }
}

template <int OP, bool RF>
cudaError_t block_dispatch(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, int pack,
                           int num, cudaStream_t st) {
    if constexpr (OP == C_TRSM) {
        return solve_cols_dispatch<64, false>(n, nrhs, A, B, batch, pack, st);
    } else if constexpr (OP == C_POTRS) {
        return solve_cols_dispatch<64, true>(n, nrhs, A, B, batch, pack, st);
    } else {
        const size_t smem = rows_team_bytes(n) * pack;
        const int grid = ceil_div(batch, pack);
        const int th = rows::T * pack;
#define GL_R(NN) (nrhs <= 1 ? launch_k(k_chol_rows<OP, NN, RF, 1>, grid, th, smem, st, n, nrhs, A, B, info, batch, num) \
                         : launch_k(k_chol_rows<OP, NN, RF, 4>, grid, th, smem, st, n, nrhs, A, B, info, batch, num))
        switch (nmax_bucket(n)) {
            case 8: return GL_R(8);
            case 16: return GL_R(16);
            case 32: return GL_R(32);
            default: return GL_R(64);
        }
#undef GL_R
    }
}

template <int OP>
size_t smem_of(int n, int nrhs, Placement pl, int refine) {
    switch (pl.scope) {
        case SCOPE_THREAD:
            return (size_t)32 * pl.pack * (odd_stride(n * n) + (has_rhs(OP) ? odd_stride(n * nrhs) : 0)) * 4;
        case SCOPE_WARP: {
            if (OP == C_TRSM) return solve_cols_per(n, nrhs, 32) * pl.pack;
            if (has_factor(OP) && n > 16) return tc_smem(n) * pl.pack;
            const int N = nmax_bucket(n);
            return (size_t)pl.pack * (N + (refine ? N * (N + 1) : 0)) * 4;
        }
        default:
            if (OP == C_TRSM || OP == C_POTRS) return solve_cols_per(n, nrhs, 64) * pl.pack;
            return rows_team_bytes(n) * pl.pack;
    }
}

template <int OP>
bool feasible_of(int n, int nrhs, Placement pl, int refine) {
    if (n < 1 || n > 64) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (pl.scope == SCOPE_THREAD && n > 16) return false;
    if (pl.scope == SCOPE_BLOCK && 64 * pl.pack > 256) return false;
    return smem_of<OP>(n, nrhs, pl, refine) <= kMaxSmem;
}

template <int OP>
cudaError_t run(int n, int nrhs, const Mat &A, const Mat &B, int *info, int batch, Placement pl, int num,
                int refine, cudaStream_t st) {
    if (!feasible_of<OP>(n, nrhs, pl, refine)) return cudaErrorInvalidConfiguration;
    if constexpr (OP == C_POSV) {
        if (refine) switch (pl.scope) {
            case SCOPE_THREAD: return thread_dispatch<OP, true>(n, nrhs, A, B, info, batch, pl.pack, num, st);
            case SCOPE_WARP: return warp_dispatch<OP, true>(n, nrhs, A, B, info, batch, pl.pack, num, st);
            default: return block_dispatch<OP, true>(n, nrhs, A, B, info, batch, pl.pack, num, st);
        }
    }
    switch (pl.scope) {
        case SCOPE_THREAD: return thread_dispatch<OP, false>(n, nrhs, A, B, info, batch, pl.pack, num, st);
        case SCOPE_WARP: return warp_dispatch<OP, false>(n, nrhs, A, B, info, batch, pl.pack, num, st);
        default: return block_dispatch<OP, false>(n, nrhs, A, B, info, batch, pl.pack, num, st);
    }
}

}  // namespace
}  // namespace glass
