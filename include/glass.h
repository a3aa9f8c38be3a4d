/*
 * glass.h -- C ABI of the GB300 (sm_103a) batched small-matrix library.
 *
 * The library computes the robotics-scale dense linear algebra and geometry
 * primitives of GLASS (arxiv 2609.28179, Sec. III-B) over large batches of
 * independent problems (n <= 64, "problems small enough to be owned by one
 * CUDA block", Sec. III-A), with the execution scope (one problem per
 * thread, per warp or per block) and the launch packing (problems per CTA)
 * chosen per call from an offline-measured placement table (Sec. III-A,
 * "architecture-specific tables"; Sec. IV-A placement sweeps).
 *
 * Common conventions (the paper fixes one convention for every scope,
 * Sec. III-A "share the same mathematical conventions and data layouts"):
 *  - Storage is FP32 unless a call says otherwise.  Every matrix is
 *    column-major: element (i,j) of problem b is X[b*sX + j*ldX + i], with
 *    ldX >= rows and sX the batch stride in ELEMENTS.  With
 *    opts->layout == GLASS_LAYOUT_INTERLEAVED32 the operands are instead
 *    stored as 32-problem interleaved blocks (see glass_to_interleaved32),
 *    ld/stride arguments are ignored and batch need not be a multiple of 32
 *    (the last block is padded by the caller's allocation).
 *  - Pointers are device pointers owned by the caller; the library keeps no
 *    pointer after a call returns.  `stream` is a cudaStream_t (0 = legacy
 *    default stream).
 *  - Calls never allocate device memory, never synchronise and never read
 *    device data on the host, so they may be recorded into a CUDA graph.
 *    Device-memory scratch, where needed, is supplied by the caller.
 *  - Argument errors (n < 1, n > 64, a null pointer with batch > 0, ld too
 *    small, a placement that is infeasible for the size) return a status
 *    synchronously and launch nothing.  batch == 0 is a no-op returning
 *    GLASS_OK.  A failed launch returns GLASS_ERR_CUDA.
 *  - Numerical failures do not fail the call: they are reported per problem
 *    in info[b] (0 = success, j+1 = column j is the first failing column),
 *    LAPACK style.  Outputs of a failed problem are unspecified.
 *  - Triangular factors are lower ('L'); the strict upper triangle of a
 *    factored or triangular operand is never used and keeps its contents.
 *  - Warp and block scopes accept the column-major layout only; the
 *    interleaved layout is served at thread scope.
 *  - No C++ exception crosses this interface.
 */
#ifndef GLASS_H
#define GLASS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *glass_stream_t; /* identical to cudaStream_t */

typedef enum {
    GLASS_OK = 0,
    GLASS_ERR_INVALID_VALUE = 1, /* bad size, stride, pointer or option */
    GLASS_ERR_UNSUPPORTED = 2,   /* valid request outside what is built (n > 64, dtype) */
    GLASS_ERR_CUDA = 3,          /* a CUDA launch or runtime call failed */
    GLASS_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    GLASS_ERR_WORKSPACE = 5      /* caller-supplied scratch too small or misaligned */
} glass_status;

typedef enum { GLASS_F32 = 0, GLASS_F64 = 1, GLASS_BF16 = 2 } glass_dtype;

/* Arithmetic of the GEMM contraction (and of Cholesky trailing updates when
 * a call accepts it).  The tensor-core modes accumulate in FP32. */
typedef enum {
    GLASS_MATH_FP32 = 0,     /* FP32 FFMA on the SIMT pipe */
    GLASS_MATH_BF16_TC = 1,  /* BF16 operands (storage dtype GLASS_BF16) */
    GLASS_MATH_TF32_TC = 2,  /* FP32 operands rounded to TF32 */
    GLASS_MATH_3XTF32_TC = 3 /* a = a_hi + a_lo split; hi*hi + hi*lo + lo*hi */
} glass_math;

typedef enum { GLASS_LAYOUT_COLMAJOR = 0, GLASS_LAYOUT_INTERLEAVED32 = 1 } glass_layout;

typedef enum {
    GLASS_SCOPE_AUTO = -1,
    GLASS_SCOPE_THREAD = 0, /* one problem per thread, 32*pack problems per CTA */
    GLASS_SCOPE_WARP = 1,   /* one problem per warp, pack warps per CTA        */
    GLASS_SCOPE_BLOCK = 2   /* one problem per team of threads, pack teams/CTA */
} glass_scope;

/* Operation identifiers of the placement table (the six swept operations
 * plus the split Cholesky calls). */
typedef enum {
    GLASS_OP_GEMM = 0,
    GLASS_OP_POSV = 1,        /* potrf + potrs fused */
    GLASS_OP_TRSM = 2,
    GLASS_OP_GETRF_GETRS = 3,
    GLASS_OP_ROT3 = 4,
    GLASS_OP_SE3 = 5,
    GLASS_OP_POTRF = 6,
    GLASS_OP_POTRS = 7,
    GLASS_NUM_OPS = 8
} glass_op;

typedef struct {
    int scope; /* glass_scope */
    int pack;  /* 0 = auto, else 1, 2, 4 or 8 */
} glass_placement;

typedef struct {
    int dtype;        /* glass_dtype of the stored operands (A/B of a GEMM) */
    int math;         /* glass_math */
    int layout;       /* glass_layout */
    glass_placement placement;
    int refine_steps; /* posv only: iterative-refinement steps (0 or 1) */
    int fp64_diag;    /* Cholesky: FP64 sqrt/reciprocal of the diagonal */
    int use_learned;  /* auto placement: consult the learned cost model for
                         shapes outside the measured grid */
} glass_opts;

/* ---------------------------------------------------------------- BLAS-3 */

/* Batched GEMM, C_b = A_b * B_b (beta = 0).  Sec. III-B (BLAS L1-L3);
 * Sec. IV-D (the GEMM family measured against host-batched libraries).
 * A is m x k (lda >= m), B is k x n (ldb >= k), C is m x n (ldc >= m),
 * 1 <= m, n, k <= 64.  With opts->math != FP32 the contraction runs on the
 * tensor cores: GLASS_MATH_BF16_TC requires opts->dtype == GLASS_BF16 (A and
 * B stored as bfloat16, C as FP32); the TF32 modes read FP32 A and B.
 * Tensor-core modes require m = n = k in {16, 32, 64}, packed colmajor. */
glass_status glass_batched_gemm(int m, int n, int k,
                                const void *A, int lda, long long sA,
                                const void *B, int ldb, long long sB,
                                void *C, int ldc, long long sC,
                                int batch, const glass_opts *opts, glass_stream_t stream);

/* ------------------------------------------------------------- Cholesky */

/* Batched Cholesky factorization A_b = L_b L_b^T (lower, in place).
 * Sec. III-B ("factorizations"); POTRF is a measured destructive op of
 * Sec. IV-A/IV-D.  A: n x n SPD, overwritten by L in its lower triangle.
 * info: device int[batch]. */
glass_status glass_batched_potrf(int n, void *A, int lda, long long sA, int *info,
                                 int batch, const glass_opts *opts, glass_stream_t stream);

/* Batched solve L L^T X = B with the factor from glass_batched_potrf.
 * Sec. III-B ("linear solves").  B: n x nrhs, overwritten by X. */
glass_status glass_batched_potrs(int n, int nrhs, const void *L, int lda, long long sA,
                                 void *B, int ldb, long long sB,
                                 int batch, const glass_opts *opts, glass_stream_t stream);

/* Batched SPD solve, fused factor + solve kept on chip (glass::posv of
 * Sec. III-A; POSV of Sec. IV-D).  A is overwritten by L (lower), B by X.
 * With opts->refine_steps == 1 the residual r = b - A x0 is formed in FP64
 * from the original A (re-read before L is written back) and one correction
 * dx = solve(L, r) is added, x1 = x0 + dx, for every right-hand side;
 * opts->fp64_diag computes the diagonal square roots and reciprocals in
 * FP64.  nrhs == 0 factors only. */
glass_status glass_batched_posv(int n, int nrhs, void *A, int lda, long long sA,
                                void *B, int ldb, long long sB, int *info,
                                int batch, const glass_opts *opts, glass_stream_t stream);

/* Batched triangular solve L X = B: left side, lower, no transpose,
 * non-unit diagonal.  Sec. III-B ("triangular ... updates", TRSV/TRSM of
 * the placement sweep, Sec. IV-A/IV-B).  The strict upper triangle of L is
 * not read.  B: n x nrhs, overwritten by X. */
glass_status glass_batched_trsm(int n, int nrhs, const void *L, int lda, long long sA,
                                void *B, int ldb, long long sB,
                                int batch, const glass_opts *opts, glass_stream_t stream);

/* ------------------------------------------------------------------- LU */

/* Batched LU with partial pivoting followed by the solve (Sec. III-B
 * "factorizations, and linear solves").  Pivot: the largest |a_ij| on or
 * below the diagonal of column j, the smallest row index on ties.
 * A (n x n) is overwritten by the packed factors (unit L strictly below the
 * diagonal, U on and above); ipiv: device int[batch*n], 0-based
 * sequential-swap form (rows j and ipiv[b*n+j] were exchanged at step j);
 * B (n x nrhs) is overwritten by X; info as for potrf (an exactly zero
 * pivot).  nrhs may be 0 (factor only). */
glass_status glass_batched_getrf_getrs(int n, int nrhs, void *A, int lda, long long sA,
                                       int *ipiv, void *B, int ldb, long long sB,
                                       int *info, int batch, const glass_opts *opts,
                                       glass_stream_t stream);

/* ------------------------------------------------------------- geometry */

/* Batched rotation-chain composition (Sec. III-B, SO(3) maps).  Problem b
 * holds `chain` 3x3 column-major rotations back to back at Rs + b*sRs
 * (9 floats each); R + b*sR receives R_0 R_1 ... R_{chain-1} (R_{chain-1}
 * acts first).  1 <= chain <= 64. */
glass_status glass_batched_rot3_compose(int chain, const void *Rs, long long sRs,
                                        void *R, long long sR, int batch,
                                        const glass_opts *opts, glass_stream_t stream);

/* Batched SE(3) apply (Sec. III-B, SE(3) maps).  Problem b holds `chain`
 * 4x4 column-major homogeneous transforms at T + b*sT (16 floats each; the
 * bottom row is not read) composed as T = T_0 ... T_{chain-1}; every point
 * p_i of P + b*sP (3 x npts column-major: x,y,z of point i at 3i..3i+2)
 * maps to q_i = R p_i + t written at Q + b*sQ.  P and Q must not overlap.
 * 1 <= chain <= 64, npts >= 1; sT, sP, sQ in elements. */
glass_status glass_batched_se3_apply(int chain, const void *T, long long sT, int npts,
                                     const void *P, long long sP, void *Q, long long sQ,
                                     int batch, const glass_opts *opts, glass_stream_t stream);

/* ------------------------------------------------------------- layouts */

/* Convert packed column-major rows x cols problems (stride rows*cols) to the
 * 32-problem interleaved layout: element (i,j) of problem b goes to
 * dst[((b/32)*rows*cols + j*rows + i)*32 + b%32].  dst must hold
 * ceil(batch/32)*32*rows*cols floats; pad lanes are written with 0.
 * glass_from_interleaved32 is the inverse (pad lanes are not read). */
glass_status glass_to_interleaved32(int rows, int cols, const float *src, float *dst,
                                    int batch, glass_stream_t stream);
glass_status glass_from_interleaved32(int rows, int cols, const float *src, float *dst,
                                      int batch, glass_stream_t stream);

/* ----------------------------------------------------- mixed-size batch */

/* Bytes of caller scratch glass_posv_varsize needs for `batch` instances. */
size_t glass_posv_varsize_workspace(int batch);

/* Fused SPD factor + solve over `batch` instances of different orders in a
 * single persistent launch (a batching pattern the paper does not have; it
 * composes the posv primitive of Sec. III-A).  n_dev[i] in [1, 64] is the
 * order of instance i; A + offA_dev[i] holds it column-major with lda =
 * n_i, B + offB_dev[i] its n_i x nrhs right-hand sides (ldb = n_i).  Both
 * are overwritten (L, X); info[i] as for potrf.  The instances are binned
 * by order and scheduled largest first on the device; sizes are never read
 * on the host, so the call can be captured in a CUDA graph.  ws must hold
 * glass_posv_varsize_workspace(batch) bytes, 256-byte aligned.  A bounded
 * device wait that gives up is reported by glass_last_device_status. */
glass_status glass_posv_varsize(int batch, const int *n_dev, const long long *offA_dev,
                                const long long *offB_dev, int nrhs, void *A, void *B,
                                int *info, void *ws, size_t ws_bytes,
                                const glass_opts *opts, glass_stream_t stream);

/* The same mixed-size solve for callers that cannot allocate device memory
 * (a real-time loop that forbids allocation once running, or a program whose
 * device memory belongs to another allocator): the scratch lives in a fixed
 * array inside the library, one per device, sized for batch <= 65536
 * (about 260 KB, held by every GPU that loads the library until exit).
 * The paper has no counterpart of this entry point.  Arguments are those of
 * glass_posv_varsize without ws / ws_bytes; batch > 65536 returns
 * GLASS_ERR_UNSUPPORTED and launches nothing; nothing is allocated.  The
 * first call on a device looks up the array's device address, so make it
 * before any stream capture.  Every call on a device shares the array: calls
 * that overlap on the GPU race.  Each call rebuilds all the scratch it reads,
 * so earlier contents never leak into a result. */
glass_status glass_posv_varsize_noalloc(int batch, const int *n_dev, const long long *offA_dev,
                                        const long long *offB_dev, int nrhs, void *A, void *B,
                                        int *info, const glass_opts *opts, glass_stream_t stream);

/* ------------------------------------------------------------ placement */

/* The placement the library would use for (op, n, k, batch, dtype): the
 * measured table's entry for the nearest grid cell (Sec. III-A, the
 * glass::recommend advisor), or, when use_learned != 0 and the shape lies
 * off the measured grid, the argmin of the learned cost model's predicted
 * latencies.  k is nrhs (solves), chain length (geometry) or the inner size
 * (gemm). */
glass_status glass_get_placement(int op, int n, int k, int batch, int dtype,
                                 int use_learned, glass_placement *out);

/* True (1) when a placement is feasible (instantiated, fits shared memory
 * and registers) for (op, n, k), else 0 (Sec. III-A: implementations are
 * instantiated only where size and resources allow). */
int glass_placement_feasible(int op, int n, int k, glass_placement p);

/* Learned placement model: weights of the 8-64-64-12 perceptron (5516
 * floats, host memory, layout W1[64][8] b1 W2[64][64] b2 W3[12][64] b3) and
 * the feature standardisation (mean[8], std[8]).  Copied by the call. */
glass_status glass_set_learned_model(const float *weights, int nweights,
                                     const float *feat_mean, const float *feat_std);

/* ------------------------------------------------- cost model (learned) */

/* Device kernels of the learned placement model (no counterpart in the
 * paper: it measures every cell exhaustively).  The network is
 * din -> 64 -> 64 -> 12 with ReLU; weights w (device, 5516 floats for
 * din = 8) in the layout of glass_set_learned_model.
 *   glass_mlp_forward: Y[rows][12] = f(X[rows][din]).
 *   glass_mlp_loss_grad: masked MSE over (Y - T) with mask M ([rows][12]);
 *     writes dL/dw into grad (device, overwritten) and the loss into
 *     *loss_dev (device float).  ws: device scratch of
 *     glass_mlp_workspace(rows) bytes.
 *   glass_mlp_adam: one Adam step at step count t >= 1 on w with moments
 *     m, v (device, same length), all in place. */
size_t glass_mlp_workspace(int rows);
glass_status glass_mlp_forward(int din, const float *w, int rows, const float *X, float *Y,
                               glass_stream_t stream);
glass_status glass_mlp_loss_grad(int din, const float *w, int rows, const float *X,
                                 const float *T, const float *M, float *grad,
                                 float *loss_dev, void *ws, size_t ws_bytes,
                                 glass_stream_t stream);
glass_status glass_mlp_adam(int nparams, float *w, const float *grad, float *m, float *v,
                            int t, float lr, float beta1, float beta2, float eps,
                            glass_stream_t stream);

/* ----------------------------------------------------------- diagnostics */

/* Synchronises `stream`, then reads and clears the library's device status
 * word of the current device: GLASS_OK, or GLASS_ERR_TIMEOUT when a bounded
 * device-side wait gave up since the last call. */
glass_status glass_last_device_status(glass_stream_t stream);

/* Static text for a status code. */
const char *glass_status_string(glass_status s);

/* Library build identification, e.g. "glass sm_103a". */
const char *glass_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GLASS_H */
