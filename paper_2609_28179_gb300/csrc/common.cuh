// common.cuh -- internal helpers shared by the device kernels of the library.
//
// Operand addressing, cooperative HBM <-> shared-memory staging, team
// synchronisation for the three execution scopes (one problem per thread,
// per warp, per team of threads; Sec. III-A), and the launcher declarations
// used by the C ABI in capi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/glass.h"

#define GLASS_FULL_MASK 0xffffffffu

namespace glass {

enum Scope { SCOPE_THREAD = 0, SCOPE_WARP = 1, SCOPE_BLOCK = 2 };

struct Placement {
    int scope;
    int pack;
};

// A batch of rows x cols operands.  Column-major with leading dimension ld
// and batch stride s (elements), or -- layout == INTERLEAVED32 -- element
// (i,j) of problem b at ((b/32)*rows*cols + j*rows + i)*32 + b%32.
struct Mat {
    float *p;
    int ld;
    long long s;
    int rows;
    int cols;
    int layout;

    __device__ __forceinline__ long long off(int b, int i, int j) const {
        if (layout == GLASS_LAYOUT_COLMAJOR)
            return (long long)b * s + (long long)j * ld + i;
        return ((long long)(b >> 5) * rows * cols + (long long)j * rows + i) * 32 + (b & 31);
    }
    __device__ __forceinline__ float get(int b, int i, int j) const { return p[off(b, i, j)]; }
    // Column-major only (warp and block scopes accept no other layout).
    __device__ __forceinline__ float cget(int b, int i, int j) const {
        return p[(long long)b * s + (long long)j * ld + i];
    }
    __device__ __forceinline__ void cset(int b, int i, int j, float v) const {
        p[(long long)b * s + (long long)j * ld + i] = v;
    }
    __device__ __forceinline__ void set(int b, int i, int j, float v) const { p[off(b, i, j)] = v; }
    // Packed column-major: the whole batch is one contiguous array.
    __host__ __device__ __forceinline__ bool packed() const {
        return layout == GLASS_LAYOUT_COLMAJOR && ld == rows && s == (long long)rows * cols;
    }
};

// ------------------------------------------------------------- team sync
// T == 1: a lone thread; T == 32: a warp; T > 32: a named barrier shared by
// the T threads of one team (barrier 0 is left to __syncthreads).
template <int T>
__device__ __forceinline__ void team_sync(int bar_id) {
    if constexpr (T == 32) {
        __syncwarp();
    } else if constexpr (T > 32) {
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(T) : "memory");
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GLASS_FULL_MASK, v, o);
    return v;
}

// Returns p unchanged but opaque to the optimiser, so that addresses formed
// from it are not merged with earlier identical ones (an unrolled load loop
// and store loop over the same n addresses would otherwise keep all n
// pointers live across the whole computation).
template <typename T>
__device__ __forceinline__ T *opaque(T *p) {
    asm volatile("" : "+l"(p));
    return p;
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only): every
// thread can keep many copies in flight without holding registers.  Both
// addresses must be 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
// 4-byte form (through L1): any float-aligned element, so strided and
// unaligned operands can be staged without registers as well.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Shared-memory pitch (floats) of a column of n values read with 16-byte
// loads, one column per thread: a multiple of 4 whose number of float4s is
// odd, so 8 consecutive threads hit 8 distinct 16-byte bank groups.
__host__ __device__ __forceinline__ int col_pitch(int n) {
    int p = (n + 3) & ~3;
    if (((p >> 2) & 1) == 0) p += 4;
    return p;
}

// Odd per-problem stride in shared memory: problem t's element e sits at
// t*S + e, so 32 threads reading the same e hit 32 distinct banks.
__host__ __device__ __forceinline__ int odd_stride(int per) { return per | 1; }

// q = e / d, r = e % d for 0 <= e < 2^24 using a float reciprocal and one
// correction step (exact: the fractional distance to the next integer is at
// least 1/d, far above the float rounding of e * (1/d) at these sizes).
__device__ __forceinline__ void divmod_small(int e, int d, float inv_d, int &q, int &r) {
    q = __float2int_rz(((float)e + 0.5f) * inv_d);
    r = e - q * d;
    if (r < 0) { --q; r += d; }
    else if (r >= d) { ++q; r -= d; }
}

// --------------------------------------------------------------- staging
// Copy problems b0 .. b0+cnt-1 of M (rows x cols each, column-major layout)
// into shared memory, problem p at sm + p*S, column-major with leading
// dimension `rows`.  Every element is one 4-byte cp.async copy (consecutive
// threads copy consecutive elements: 128 coalesced bytes per warp for a
// packed batch), all of a thread's copies in flight at once, so a CTA pays
// one memory round trip however many problems it stages (a register-staged
// loop waits once per few loads, which dominates when a few warps per SM
// stage many small problems).  All threads of the CTA take part; the copies
// are complete for this thread on return, and the caller synchronises the
// CTA afterwards.
__device__ __forceinline__ void stage_in(float *sm, int S, const Mat &M, int b0, int cnt) {
    const int per = M.rows * M.cols;
    const int total = cnt * per;
    const int T = blockDim.x;
    // element e = p * per + q of the staged range, advanced by T per copy
    int p = threadIdx.x / per, q = threadIdx.x - p * per;
    const int dp = T / per, dq = T - dp * per;
    if (M.packed()) {
        const float *g = M.p + (long long)b0 * per;
        for (int e = threadIdx.x; e < total; e += T) {
            cp_async4(sm + p * S + q, g + e);
            p += dp;
            q += dq;
            if (q >= per) { q -= per; ++p; }
        }
    } else {
        for (int e = threadIdx.x; e < total; e += T) {
            const int j = q / M.rows, i = q - j * M.rows;
            cp_async4(sm + p * S + q, M.p + (long long)(b0 + p) * M.s + (long long)j * M.ld + i);
            p += dp;
            q += dq;
            if (q >= per) { q -= per; ++p; }
        }
    }
    cp_async_wait_all();
}

// Inverse of stage_in: write the staged problems back to M.
__device__ __forceinline__ void stage_out(const float *sm, int S, const Mat &M, int b0, int cnt) {
    const int per = M.rows * M.cols;
    const int total = cnt * per;
    const float inv = 1.0f / (float)per;
    if (M.packed()) {
        float *g = M.p + (long long)b0 * per;
        if ((reinterpret_cast<uintptr_t>(g) & 15) == 0) {
            const int nv = total >> 2;
            float4 *g4 = reinterpret_cast<float4 *>(g);
            for (int v = threadIdx.x; v < nv; v += blockDim.x) {
                int p, q;
                divmod_small(v * 4, per, inv, p, q);
                float xs[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    xs[u] = sm[p * S + q];
                    if (++q == per) { q = 0; ++p; }
                }
                __stcs(g4 + v, make_float4(xs[0], xs[1], xs[2], xs[3]));
            }
            for (int e = (nv << 2) + threadIdx.x; e < total; e += blockDim.x) {
                int p, q;
                divmod_small(e, per, inv, p, q);
                __stcs(g + e, sm[p * S + q]);
            }
        } else {
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                int p, q;
                divmod_small(e, per, inv, p, q);
                __stcs(g + e, sm[p * S + q]);
            }
        }
    } else {
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int p, q;
            divmod_small(e, per, inv, p, q);
            const int j = q / M.rows, i = q - j * M.rows;
            M.set(b0 + p, i, j, sm[p * S + q]);
        }
    }
}

// Diagonal square root and reciprocal of a Cholesky pivot d > 0, in FP32 or
// (fp64 == true) to FP64 accuracy rounded once to FP32 -- the values an FP64
// square root and division give, without FP64 operations, which GB300's
// narrow FP64 pipe makes costly (every lane would issue them per column):
//  - the FP64 square root rounded to FP32 is sqrtf(d) itself (a 53-bit
//    square root rounds to the correctly rounded 24-bit one, 53 >= 2*24+2);
//  - 1/sqrt(d) = (1/l)(1 + t)^(-1/2) with t = (d - l^2)/l^2, and 1/l =
//    r0 / (1 - eps) with eps = 1 - l r0, r0 the rounded reciprocal; both
//    remainders are exact in FP32 by one fused multiply-add (Markstein), so
//    1/sqrt(d) = r0 (1 + eps - t/2) up to terms of order 2^-46, formed as
//    r0 + r0 (eps - t/2) and rounded once: the FP64 result except within
//    about 2^-46 of a rounding boundary.
__device__ __forceinline__ void chol_diag(float d, bool fp64, float &l, float &r) {
    l = sqrtf(d);
    const float r0 = __frcp_rn(l);  // the correctly rounded 1 / l
    if (fp64) {
        const float e = fmaf(-l, l, d);       // d - l^2, exact
        const float eps = fmaf(-l, r0, 1.0f);  // 1 - l r0, exact
        const float t = e * r0 * r0;           // (d - l^2) / l^2, |t| < 2^-22
        r = fmaf(r0, fmaf(-0.5f, t, eps), r0);
    } else {
        r = r0;
    }
}

// Numerics flags of the Cholesky launchers and kernels (the `num` argument):
// the FP64-accurate diagonal, and the compensated FP32 refinement residual
// instead of the FP64 one.
constexpr int NUM_FP64_DIAG = 1;
constexpr int NUM_DOT2_RESIDUAL = 2;

// Compensated accumulation of s = b - sum_k a_k x_k in FP32 (Ogita, Rump and
// Oishi, "Accurate sum and dot product", 2005, algorithm Dot2): each product
// is split exactly into p + e (p = fl(a x), e = fma(a, x, -p): Dekker's
// TwoProduct with a fused multiply-add) and each addition into t + q
// (Knuth's TwoSum, six additions, no branch); the errors e and q are summed
// in c, and s + c carries the result as if computed in twice the working
// precision.  The _rn intrinsics keep the compiler from contracting the
// products and sums into fused multiply-adds, which would lose the exact
// splits.
struct Dot2 {
    float s, c;
    __device__ __forceinline__ void init(float b) {
        s = b;
        c = 0.f;
    }
    __device__ __forceinline__ void sub(float a, float x) {  // s -= a x
        const float p = __fmul_rn(-a, x);
        const float e = fmaf(-a, x, -p);
        const float t = __fadd_rn(s, p);
        const float z = __fadd_rn(t, -s);
        const float q = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -z)), __fadd_rn(p, -z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(q, e));
    }
    // Merges another partial sum (TwoSum of the leading parts).
    __device__ __forceinline__ void merge(const Dot2 &o) {
        const float t = __fadd_rn(s, o.s);
        const float z = __fadd_rn(t, -s);
        const float q = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -z)), __fadd_rn(o.s, -z));
        s = t;
        c = __fadd_rn(__fadd_rn(c, o.c), q);
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};

// FP32 -> FP64 conversion on the integer pipe, without branches: for a
// normal value the sign moves to bit 63, the 8-bit exponent is rebiased from
// 127 to 1023 and the 23-bit fraction becomes the top of the 52-bit one
// (exact); zeros keep their sign, infinities and NaNs (payload included)
// stay infinities and NaNs, subnormals become zero of the same sign (an
// absolute change below 2^-126).  On GB300 the FP64 pipe is narrow, and the
// hardware conversion would occupy it as much as the fused multiply-add
// that uses the value.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e8 = (u >> 23) & 0xffu;
    const unsigned e11 = e8 == 0u ? 0u : (e8 == 0xffu ? 0x7ffu : e8 + 896u);
    const unsigned m = e8 == 0u ? 0u : (u & 0x7fffffu);
    return __hiloint2double((int)((u & 0x80000000u) | (e11 << 20) | (m >> 3)), (int)(m << 29));
}

// ------------------------------------------------------- launch helpers
// Raise a kernel's dynamic shared-memory limit to at least `bytes` once per
// (device, kernel); later calls are a lookup, so launches recorded into a
// CUDA graph never call into the runtime's attribute API.
cudaError_t prepare_kernel(const void *fn, size_t bytes);

template <typename K>
inline cudaError_t prepare(K kern, size_t bytes) {
    return bytes > 48 * 1024 ? prepare_kernel(reinterpret_cast<const void *>(kern), bytes) : cudaSuccess;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Problems per CTA and threads per CTA of a placement for a team size T.
struct Geometry {
    int per_cta;   // problems per CTA
    int threads;   // threads per CTA
    int grid;      // CTAs
};

// --------------------------------------------------- launchers (by file)
// Each returns cudaSuccess or the launch error; none allocates or syncs.
// k_chol.cu
cudaError_t launch_potrf(int n, Mat A, int *info, int batch, Placement pl, int num,
                         cudaStream_t st);
cudaError_t launch_potrs(int n, int nrhs, Mat L, Mat B, int batch, Placement pl, cudaStream_t st);
cudaError_t launch_trsm(int n, int nrhs, Mat L, Mat B, int batch, Placement pl, cudaStream_t st);
cudaError_t launch_posv(int n, int nrhs, Mat A, Mat B, int *info, int batch, Placement pl,
                        int num, int refine, cudaStream_t st);  // num: NUM_* flags
size_t smem_chol(int op, int n, int nrhs, Placement pl);
bool feasible_chol(int op, int n, int nrhs, Placement pl);
// k_lu.cu
cudaError_t launch_getrf_getrs(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch,
                               Placement pl, cudaStream_t st);
bool feasible_lu(int n, int nrhs, Placement pl);
// k_gemm.cu
cudaError_t launch_gemm(int m, int n, int k, Mat A, Mat B, Mat C, int batch, Placement pl,
                        cudaStream_t st);
bool feasible_gemm(int m, int n, int k, Placement pl);
// k_gemm_tc.cu
cudaError_t launch_gemm_tc(int n, int math, const void *A, const void *B, float *C, int batch,
                           cudaStream_t st);
// Order-64 products on the fifth-generation tensor cores (3xTF32 split),
// contiguous 16-byte aligned batches only.
cudaError_t launch_gemm_umma64(const float *A, const float *B, float *C, int batch, cudaStream_t st);
// The same with an explicit wait limit (clock cycles) and, for a test of the
// bounded-wait path, the kernel's bulk copies withheld.
cudaError_t launch_gemm_umma64_ex(const float *A, const float *B, float *C, int batch, long long wait_cycles,
                                  int withhold_loads, cudaStream_t st);
// capi.cu: the device status word of the current device (bounded device-side
// waits that gave up record GLASS_ERR_TIMEOUT there), or null.
unsigned *device_status_word();
// k_geom.cu
cudaError_t launch_rot3(int chain, Mat Rs, Mat R, int batch, Placement pl, cudaStream_t st);
cudaError_t launch_se3(int chain, Mat T, int npts, Mat P, Mat Q, int batch, Placement pl,
                       cudaStream_t st);
bool feasible_geom(int op, int chain, Placement pl);
cudaError_t launch_to_interleaved(int rows, int cols, const float *src, float *dst, int batch,
                                  cudaStream_t st);
cudaError_t launch_from_interleaved(int rows, int cols, const float *src, float *dst, int batch,
                                    cudaStream_t st);
// k_varsize.cu
size_t varsize_workspace(int batch);
cudaError_t launch_posv_varsize(int batch, const int *n_dev, const long long *offA,
                                const long long *offB, int nrhs, float *A, float *B, int *info,
                                void *ws, int warps_per_cta, unsigned *status, cudaStream_t st);
// k_riccati.cu
bool feasible_gemm_ex(int ta, int tb, int m, int n, int k, Placement pl);
cudaError_t launch_gemm_ex(int ta, int tb, int m, int n, int k, float alpha, Mat A, Mat B, float beta, Mat C,
                           int batch, Placement pl, cudaStream_t st);
size_t riccati_floats(int nx, int nu);
bool feasible_riccati(int nx, int nu, Placement pl);
cudaError_t launch_riccati(int nx, int nu, const float *A, long long sA, const float *B, long long sB,
                           const float *P, long long sP, const float *R, long long sR, float *K, long long sK,
                           int *info, int batch, Placement pl, cudaStream_t st);
// k_robo.cu (op = glass_robo_op)
enum RoboOp {
    ROBO_QUAT_RETRACT = GLASS_ROBO_QUAT_RETRACT,
    ROBO_QUAT_ERROR = GLASS_ROBO_QUAT_ERROR,
    ROBO_SE3_RETRACT = GLASS_ROBO_SE3_RETRACT,
    ROBO_MOTION_CROSS = GLASS_ROBO_MOTION_CROSS,
    ROBO_EIG3 = GLASS_ROBO_EIG3,
    ROBO_SVD3 = GLASS_ROBO_SVD3,
    ROBO_CLOSEST_ROTATION = GLASS_ROBO_CLOSEST_ROTATION,
    ROBO_ARGMAX = GLASS_ROBO_ARGMAX,
    ROBO_SOFTMAX = GLASS_ROBO_SOFTMAX
};
bool feasible_robo(int op, int n, Placement pl);
cudaError_t launch_robo(int op, int n, const float *a, const float *b, long long sa, float *o1, float *o2, float *o3,
                        long long so, int *idx, int batch, Placement pl, cudaStream_t st);
// k_blas.cu
cudaError_t launch_dot(int n, const float *x, long long sx, const float *y, long long sy, float *out, int batch,
                       Placement pl, cudaStream_t st);
cudaError_t launch_gemv(int trans, int m, int n, float alpha, Mat A, const float *x, long long sx, float beta, float *y,
                        long long sy, int batch, Placement pl, cudaStream_t st);
cudaError_t launch_btd_matvec(int nb, int N, const float *D, const float *O, const float *x, float *y, int batch,
                              int pack, cudaStream_t st);
cudaError_t launch_btd_posv(int nb, int N, float *D, float *O, float *bx, int *info, int batch, int pack,
                            cudaStream_t st);
size_t btd_pcg_smem(int nb, int N, int pack);
cudaError_t launch_btd_pcg(int nb, int N, const float *D, const float *O, const float *b, float *x, int iters,
                           float tol, int *done, float *ws, int batch, int pack, cudaStream_t st);
// k_fp64.cu (op = glass_op)
bool feasible_f64(int op, int n, Placement pl);
cudaError_t launch_gemm_f64(int m, int n, int k, const double *A, int lda, long long sA, const double *B, int ldb,
                            long long sB, double *C, int ldc, long long sC, int batch, Placement pl, cudaStream_t st);
cudaError_t launch_chol_f64(int op, int n, int nrhs, double *A, int lda, long long sA, double *B, int ldb, long long sB,
                            int *info, int batch, Placement pl, cudaStream_t st);
cudaError_t launch_lu_f64(int n, int nrhs, double *A, int lda, long long sA, int *ipiv, double *B, int ldb, long long sB,
                          int *info, int batch, Placement pl, cudaStream_t st);
// k_mlp.cu
size_t mlp_workspace(int rows);
cudaError_t launch_mlp_forward(int din, const float *w, int rows, const float *X, float *Y,
                               cudaStream_t st);
cudaError_t launch_mlp_loss_grad(int din, const float *w, int rows, const float *X,
                                 const float *T, const float *M, float *grad, float *loss,
                                 void *ws, cudaStream_t st);
cudaError_t launch_mlp_adam(int np, float *w, const float *g, float *m, float *v, int t,
                            float lr, float b1, float b2, float eps, cudaStream_t st);

}  // namespace glass
