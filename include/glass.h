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

/* Arithmetic of the refinement residual r = b - A x0 (posv with
 * refine_steps == 1).  GLASS_RESIDUAL_FP64 accumulates in FP64.
 * GLASS_RESIDUAL_DOT2 accumulates on the FP32 pipe with error-free
 * transformations (Ogita, Rump and Oishi, "Accurate sum and dot product",
 * SIAM J. Sci. Comput. 26(6), 2005, algorithm Dot2): every product's and
 * every addition's exact rounding error is carried in a second FP32 sum, so
 * r is as accurate as if it were evaluated in twice the FP32 precision and
 * then rounded -- ample for one correction of an FP32 solve, without GB300's
 * narrow FP64 pipe.  The paper prescribes neither; FP64 is the default. */
typedef enum { GLASS_RESIDUAL_FP64 = 0, GLASS_RESIDUAL_DOT2 = 1 } glass_residual;

typedef enum {
    GLASS_SCOPE_AUTO = -1,
    GLASS_SCOPE_THREAD = 0, /* one problem per thread, 32*pack problems per CTA */
    GLASS_SCOPE_WARP = 1,   /* one problem per warp, pack warps per CTA        */
    GLASS_SCOPE_BLOCK = 2,  /* one problem per team of threads, pack teams/CTA */
    GLASS_SCOPE_COMPOSED = 3 /* composite operations only: one library call per
                                primitive step, intermediates in global memory */
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
    int dtype;        /* glass_dtype of the stored operands: GLASS_F32; GLASS_BF16
                         for the A/B of a BF16 tensor-core GEMM; GLASS_F64 (the
                         paper's fp64 sweep variants) for gemm, potrf, potrs,
                         posv, trsm and getrf_getrs -- every operand, the
                         strides in doubles, thread scope (n <= 8) or warp
                         scope (n <= 64 while the packed problems fit shared
                         memory), no refinement, FP64 divisions and square
                         roots; its own measured placement table */
    int math;         /* glass_math */
    int layout;       /* glass_layout */
    glass_placement placement;
    int refine_steps; /* posv only: iterative-refinement steps (0 or 1) */
    int fp64_diag;    /* Cholesky: diagonal sqrt/reciprocal to FP64 accuracy */
    int use_learned;  /* auto placement: consult the learned cost model for
                         shapes outside the measured grid */
    int residual;     /* posv refinement: glass_residual (0 = FP64) */
} glass_opts;

/* ---------------------------------------------------------------- BLAS-3 */

/* Batched GEMM, C_b = A_b * B_b (beta = 0).  Sec. III-B (BLAS L1-L3);
 * Sec. IV-D (the GEMM family measured against host-batched libraries).
 * A is m x k (lda >= m), B is k x n (ldb >= k), C is m x n (ldc >= m),
 * 1 <= m, n, k <= 64.  With opts->math != FP32 the contraction runs on the
 * tensor cores: GLASS_MATH_BF16_TC requires opts->dtype == GLASS_BF16 (A and
 * B stored as bfloat16, C as FP32); the TF32 modes read FP32 A and B.
 * Tensor-core modes require m = n = k in {16, 32, 64}, packed colmajor.
 * Order 64 runs on the fifth-generation tensor cores (tcgen05, operands in
 * shared memory, accumulator in tensor memory) in the BF16 and 3xTF32 modes
 * and for the FP32 block-scope placement (pack 1) with packed, 16-byte
 * aligned operands; the split-TF32 kernel also adds the lo*lo product, and
 * its error stays within the FP32 bound 2 k u |A||B|.  Those kernels' waits
 * are bounded: one that gives up records GLASS_ERR_TIMEOUT for
 * glass_last_device_status. */
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
 * (or, with opts->residual == GLASS_RESIDUAL_DOT2, as a compensated FP32
 * dot product) from the original A (re-read before L is written back) and
 * one correction
 * dx = solve(L, r) is added, x1 = x0 + dx, for every right-hand side;
 * opts->fp64_diag computes the diagonal square roots and reciprocals to
 * FP64 accuracy, each rounded once to FP32 (the square root is the FP32 one,
 * which equals the rounded FP64 square root; the reciprocal is corrected by
 * its exact FP32 remainders, so GB300's narrow FP64 pipe is not needed).
 * nrhs == 0 factors only. */
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
 * GLASS_ERR_UNSUPPORTED and launches nothing; nothing is allocated.  Every
 * call looks up the array's device address on the current device (so a
 * context destroyed and re-created in between is handled); the first call on
 * a device may also load the library's device code there, so make that first
 * call before any stream capture.  Every call on a device shares the array: calls
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

/* ------------------------------------------------- composite operations */

/* Batched GEMM with operand transposes and scaling (Sec. III-B "BLAS
 * L1-L3"; the BLAS xGEMM contract):
 *   C = alpha op(A) op(B) + beta C,  op(X) = X (trans 0) or X^T (trans 1),
 * C m x n, op(A) m x k, op(B) k x n, 1 <= m, n, k <= 64, FP32, column-major
 * with leading dimensions of the STORED operands (A is k x m when transa).
 * With beta == 0, C is not read.  Placement: warp (one warp per problem) or
 * block (a 128-thread team), pack problems per CTA; auto picks by size.
 * Operands are staged in shared memory with cp.async. */
glass_status glass_batched_gemm_ex(int transa, int transb, int m, int n, int k, float alpha,
                                   const void *A, int lda, long long sA, const void *B, int ldb,
                                   long long sB, float beta, void *C, int ldc, long long sC,
                                   int batch, const glass_opts *opts, glass_stream_t stream);

/* LQR feedback gain (Sec. III-B fused operations; Sec. IV-E, Fig. 7):
 *   K = (R + B^T P B)^{-1} B^T P A
 * A nx x nx, B nx x nu, P nx x nx (symmetric: the cost-to-go of the
 * Riccati recursion), R nu x nu (symmetric positive definite), K nu x nx;
 * 1 <= nx, nu <= 64; FP32, each operand packed column-major (leading
 * dimension = rows) with batch stride s* in elements (inputs may use 0).
 * info[b] is the Cholesky info of S = R + B^T P B (0, or j+1 for the first
 * failing column; K is unspecified then).
 * Two placements compute it (fusion granularity is itself a placement,
 * Sec. IV-E): a fused kernel (scope warp or block, pack problems per CTA)
 * that keeps P B, S, B^T P A and the factor of S in shared memory, or the
 * composition (scope GLASS_SCOPE_COMPOSED) of glass_batched_gemm (P B),
 * one device copy (S = R), glass_batched_gemm_ex (S += B^T (P B);
 * K = (P B)^T A) and glass_batched_posv (K = S^{-1} K), intermediates in the
 * caller's workspace ws of at least glass_riccati_workspace(nx, nu, batch)
 * bytes (256-byte aligned).  Both form B^T P A as (P B)^T A.  Auto resolves
 * from a measured table; the composition is chosen only when ws is large
 * enough, and requesting it without that workspace is GLASS_ERR_WORKSPACE. */
size_t glass_riccati_workspace(int nx, int nu, int batch);
glass_status glass_riccati_gain(int nx, int nu, const void *A, long long sA, const void *B,
                                long long sB, const void *P, long long sP, const void *R,
                                long long sR, void *K, long long sK, int *info, int batch,
                                void *ws, size_t ws_bytes, const glass_opts *opts,
                                glass_stream_t stream);

/* The placement glass_riccati_gain resolves for (nx, nu, batch) when the
 * composition is (composed_ok != 0) or is not available. */
glass_status glass_riccati_placement(int nx, int nu, int batch, int composed_ok,
                                     glass_placement *out);
/* 1 when the fused kernel can run (nx, nu) at placement p, else 0. */
int glass_riccati_feasible(int nx, int nu, glass_placement p);

/* ------------------------------------------------- robotics operations */

/* The robotics operations of the paper's placement table (Sec. IV-E,
 * Table II).  Conventions (the paper
 * requires an operation's interface to fix them, Sec. III-B):
 *  - quaternion q = (w, x, y, z), Hamilton product, unit norm expected;
 *  - rotation vector d: angle |d| about d / |d|, Exp(d) = (cos |d|/2,
 *    sin(|d|/2) d / |d|), Log its inverse on the w >= 0 hemisphere;
 *  - retractions perturb on the right: quat_retract(q, d) = q Exp(d),
 *    se3_retract(T, xi) = T Exp(xi); quat_error(q1, q2) = Log(q1^-1 q2);
 *  - twists xi and motion vectors are (linear, angular);
 *    motion_cross(v, m) = v x m = (w x m_lin + v_lin x m_ang, w x m_ang),
 *    w = v_ang;
 *  - 4x4 homogeneous transforms and 3x3 matrices are column-major; the
 *    bottom row of an input transform is not read, outputs get (0 0 0 1);
 *  - eig3 (symmetric A): eigenvalues ascending, eigenvector columns with
 *    their largest-magnitude component positive; only the lower triangle is
 *    not enough -- all nine entries are read and A must be symmetric;
 *  - svd3: M = U diag(s) V^T, s descending, s >= 0, U and V orthogonal;
 *  - closest_rotation(M) = U diag(1, 1, det(U V^T)) V^T, the rotation
 *    nearest M in the Frobenius norm;
 *  - argmax: the first index of the largest of n values (NaN inputs
 *    unspecified); softmax: exp(x_i - max) / sum_j exp(x_j - max).
 * Storage is FP32, problem b's operands packed at b times their size
 * (q: 4, d: 3, T: 16, xi: 6, v/m: 6, 3x3: 9, eigen/singular values: 3);
 * quaternion and transform arrays must be 16-byte aligned.  argmax and
 * softmax read x[b*sx + i], i < n, and write idx[b] / y[b*sy + i].
 * Placement: scope thread (one problem per thread, 32*pack per CTA); argmax
 * and softmax also warp (one problem per warp) or block (a 64-thread team,
 * pack <= 4), the n values spread over the team; auto resolves from the
 * measured table.  The seven element-wise operations accept thread scope
 * only (a warp or block placement returns GLASS_ERR_INVALID_VALUE): a
 * problem is a short serial chain with nothing for a team to share. */
typedef enum {
    GLASS_ROBO_QUAT_RETRACT = 0,
    GLASS_ROBO_QUAT_ERROR = 1,
    GLASS_ROBO_SE3_RETRACT = 2,
    GLASS_ROBO_MOTION_CROSS = 3,
    GLASS_ROBO_EIG3 = 4,
    GLASS_ROBO_SVD3 = 5,
    GLASS_ROBO_CLOSEST_ROTATION = 6,
    GLASS_ROBO_ARGMAX = 7,
    GLASS_ROBO_SOFTMAX = 8,
    GLASS_ROBO_NUM_OPS = 9
} glass_robo_op;

glass_status glass_batched_quat_retract(const void *q, const void *d, void *out, int batch,
                                        const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_quat_error(const void *q1, const void *q2, void *out, int batch,
                                      const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_se3_retract(const void *T, const void *xi, void *out, int batch,
                                       const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_motion_cross(const void *v, const void *m, void *out, int batch,
                                        const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_eig3(const void *A, void *w, void *V, int batch,
                                const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_svd3(const void *M, void *U, void *s, void *V, int batch,
                                const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_closest_rotation(const void *M, void *R, int batch,
                                            const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_argmax(int n, const void *x, long long sx, int *idx, int batch,
                                  const glass_opts *opts, glass_stream_t stream);
glass_status glass_batched_softmax(int n, const void *x, long long sx, void *y, long long sy,
                                   int batch, const glass_opts *opts, glass_stream_t stream);

/* The placement the robotics operation `op` resolves at `batch` (n: the
 * length for argmax/softmax, else ignored), and its feasibility test. */
glass_status glass_robo_placement(int op, int n, int batch, glass_placement *out);
int glass_robo_feasible(int op, int n, glass_placement p);

/* ----------------------------------------- BLAS-1/2, block-tridiagonal */

/* Batched dot product (Sec. III-B reductions, BLAS L1):
 * out[b] = sum_{i<n} x[b*sx + i] y[b*sy + i], n >= 1.  Placement: thread
 * (one problem per thread), warp or block (64 threads) with a shuffle
 * reduction; auto picks by n. */
glass_status glass_batched_dot(int n, const void *x, long long sx, const void *y, long long sy,
                               void *out, int batch, const glass_opts *opts, glass_stream_t stream);

/* Batched GEMV (BLAS L2): y = alpha op(A) x + beta y, A m x n column-major
 * (lda >= m, batch stride sA), op(A) = A (trans 0: x has n entries, y m) or
 * A^T (trans 1: x m, y n); 1 <= m, n <= 64; beta == 0 does not read y.
 * Placement: thread or warp (rows over lanes); auto picks by size. */
glass_status glass_batched_gemv(int trans, int m, int n, float alpha, const void *A, int lda,
                                long long sA, const void *x, long long sx, float beta, void *y,
                                long long sy, int batch, const glass_opts *opts,
                                glass_stream_t stream);

/* Batched triangular solve with one right-hand side (BLAS L2 TRSV: left,
 * lower, no transpose, non-unit): L x = b, x overwrites b (x[b*sx + i]).
 * The trsm kernels with nrhs = 1 and the trsm placement table. */
glass_status glass_batched_trsv(int n, const void *L, int lda, long long sA, void *x, long long sx,
                                int batch, const glass_opts *opts, glass_stream_t stream);

/* Symmetric block-tridiagonal operators of trajectory optimization (Sec.
 * III-B structured routines): T has N >= 1 diagonal blocks D_i and N-1
 * sub-diagonal blocks O_i = T[i+1][i] (the super-diagonal blocks are their
 * transposes), each nb x nb column-major (1 <= nb <= 32), packed per
 * problem: D [batch][N][nb*nb], O [batch][N-1][nb*nb], vectors
 * [batch][N*nb].  One warp per problem (pack warps per CTA).
 *   btd_matvec: y = T x (every entry of D_i is read).
 *   btd_posv:   T x = b for SPD T by the block Cholesky recurrence
 *     L_0 L_0^T = D_0, W_i = O_i L_i^{-T}, L_{i+1} L_{i+1}^T = D_{i+1} -
 *     W_i W_i^T, then the block forward and backward sweeps; in place:
 *     D_i <- L_i (lower triangle; the strict upper triangle keeps its
 *     contents), O_i <- W_i, b <- x.  info[b] = 0, or i*nb + j + 1 when the
 *     j-th column of block i fails (the global column of the dense
 *     Cholesky of T). */
glass_status glass_batched_btd_matvec(int nb, int N, const void *D, const void *O, const void *x,
                                      void *y, int batch, const glass_opts *opts,
                                      glass_stream_t stream);
glass_status glass_batched_btd_posv(int nb, int N, void *D, void *O, void *b, int *info, int batch,
                                    const glass_opts *opts, glass_stream_t stream);

/* Iterative solve of the same T x = b (Sec. III-B names direct and
 * iterative solvers for these operators; the method is the reading of this
 * library): preconditioned conjugate gradient with the block-Jacobi
 * preconditioner M = blockdiag(D_0, ..., D_{N-1}).  r = b - T x, z = M^{-1}
 * r, p = z, rho = r'z, rho0 = rho; while k < iters and rho > tol^2 rho0 (and
 * rho > 0): q = T p, alpha = rho / p'q (the loop also ends when p'q <= 0),
 * x += alpha p, r -= alpha q, z = M^{-1} r, p = z + (r'z / rho) p, k += 1.
 * tol = 0 runs exactly `iters` iterations on an SPD T.  x [batch][N*nb]
 * holds the initial guess on entry and the last iterate on return (warm
 * starts); b [batch][N*nb] is read only; D and O as above, read only.
 * iters_done[b] (device int) receives k, or -1 when some D_i is not
 * positive definite (x is then left as given).  ws: device scratch of
 * glass_btd_pcg_workspace(nb, N, batch) bytes, 16-byte aligned (it holds
 * the D_i^{-1}); else GLASS_ERR_WORKSPACE.  1 <= nb <= 32, 1 <= N <= 64,
 * iters >= 0, tol >= 0.  One warp per problem; placement pack = warps per
 * CTA (0: up to 4 as shared memory allows). */
size_t glass_btd_pcg_workspace(int nb, int N, int batch);
glass_status glass_batched_btd_pcg(int nb, int N, const void *D, const void *O, const void *b, void *x,
                                   int iters, float tol, int *iters_done, void *ws, size_t ws_bytes,
                                   int batch, const glass_opts *opts, glass_stream_t stream);

/* ------------------------------------------------------- measurement aid */

/* Pipe-throughput probe (no counterpart in the paper; it supplies the
 * measured peaks the rooflines are quoted against).  Launches `blocks` CTAs
 * of `threads` threads (32..256, a multiple of 32) that keep one pipe busy
 * with independent work for `iters` iterations:
 *   kind 0: FP32 FFMA, 1: FP64 DFMA, 2: TF32 mma.sync m16n8k8,
 *   3: BF16 mma.sync m16n8k16 (FP32 accumulation).
 * sink: device scratch of blocks*threads elements (float; double for kind
 * 1), written only to keep the work live.  *flops (host, may be null)
 * receives the floating-point operations of one launch (an FMA counts 2).
 * Time the launch on `stream` with events; flops / time is the peak. */
glass_status glass_peak_probe(int kind, int iters, int blocks, int threads, void *sink,
                              double *flops, glass_stream_t stream);

/* ----------------------------------------------------------- diagnostics */

/* Synchronises `stream`, then reads and clears the library's device status
 * word of the current device: GLASS_OK, GLASS_ERR_TIMEOUT when a bounded
 * device-side wait gave up since the last call, or GLASS_ERR_UNSUPPORTED when
 * a tensor-core GEMM CTA found its shared memory misaligned (its C is then
 * left unwritten). */
glass_status glass_last_device_status(glass_stream_t stream);

/* Test of the bounded-wait path (the paper has no counterpart; failure
 * handling of the device-side waits above).  Launches the order-64 tcgen05
 * GEMM of glass_batched_gemm on `batch` problems (A, B, C: contiguous 64 x 64
 * FP32 batches, 16-byte aligned) with its bulk copies withheld, so that its
 * first mbarrier waits give up after wait_cycles clock cycles (1 <=
 * wait_cycles <= 2^31) with nothing in flight: the kernel then records
 * GLASS_ERR_TIMEOUT for glass_last_device_status, writes nothing to C and
 * returns, and the context stays usable.  Returns the launch status. */
glass_status glass_selftest_wait_timeout(const float *A, const float *B, float *C, int batch,
                                         long long wait_cycles, glass_stream_t stream);

/* Static text for a status code. */
const char *glass_status_string(glass_status s);

/* Library build identification, e.g. "glass sm_103a". */
const char *glass_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GLASS_H */
