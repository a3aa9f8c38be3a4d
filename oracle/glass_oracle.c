/*
 * glass_oracle.c -- plain, slow, obviously-correct FP64 reference for the
 * batched small-matrix operations of GLASS (arxiv 2609.28179).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA library
 * shares no code, header, table or helper with this file, and this file
 * includes nothing from it.
 *
 * Conventions (shared by contract, not by code, with the device library):
 *   - every matrix is column-major: element (i,j) of problem b lives at
 *     X[b*sX + j*ldX + i];
 *   - Cholesky works on the lower triangle only; the strict upper triangle is
 *     neither read nor written (LAPACK uplo='L');
 *   - info[b] = 0 on success, j+1 when column j is the first that fails
 *     (LAPACK convention);
 *   - ipiv is 0-based with sequential-swap semantics: at step j rows j and
 *     ipiv[j] were exchanged (the convention of scipy.linalg.lu_factor).
 *
 * Every routine is the textbook definition of the operation, with no
 * blocking, fusion or reordering.  The batch loop is the only parallel loop
 * (OpenMP), so results do not depend on the thread count.
 *
 * The paper names the operation classes (Sec. III-B: BLAS L1-L3, triangular
 * and symmetric updates, factorizations, linear solves; SO(3)/SE(3) maps) and
 * the measured POTRF/POSV/GEMM families (Sec. IV-A, IV-D); it prints no
 * algorithm listing, so each routine below is the standard definition.
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 0; /* 0 = OpenMP default */

void oracle_set_threads(int t) { g_threads = t; }

int oracle_max_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

#define OMP_FOR _Pragma("omp parallel for schedule(static) num_threads(oracle_max_threads())")

/* ------------------------------------------------------------------------ */
/* GEMM  C = A * B   (Sec. III-B "BLAS L1-L3"; Sec. IV-D GEMM)              */
/* A is m x k, B is k x n, C is m x n; c_ij = sum_l a_il b_lj.               */
/* ------------------------------------------------------------------------ */
void oracle_gemm_f64(int m, int n, int k,
                     const double *A, int lda, long long sA,
                     const double *B, int ldb, long long sB,
                     double *C, int ldc, long long sC, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *a = A + (long long)b * sA;
        const double *bb = B + (long long)b * sB;
        double *c = C + (long long)b * sC;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int l = 0; l < k; ++l)
                    s += a[l * lda + i] * bb[j * ldb + l];
                c[j * ldc + i] = s;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* POTRF  A = L L^T, lower, in place  (Sec. III-B factorizations; POTRF is    */
/* one of the measured destructive ops of Sec. IV-A).                        */
/*   for j: d = a_jj - sum_{k<j} l_jk^2 ; d <= 0 or NaN -> info = j+1, stop  */
/*          l_jj = sqrt(d) ; l_ij = (a_ij - sum_{k<j} l_ik l_jk) / l_jj      */
/* ------------------------------------------------------------------------ */
static int potrf_one(int n, double *a, int lda)
{
    for (int j = 0; j < n; ++j) {
        double d = a[j * lda + j];
        for (int k = 0; k < j; ++k)
            d -= a[k * lda + j] * a[k * lda + j];
        if (!(d > 0.0))            /* also catches NaN */
            return j + 1;
        double ljj = sqrt(d);
        a[j * lda + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = a[j * lda + i];
            for (int k = 0; k < j; ++k)
                s -= a[k * lda + i] * a[k * lda + j];
            a[j * lda + i] = s / ljj;
        }
    }
    return 0;
}

void oracle_potrf_f64(int n, double *A, int lda, long long sA, int *info, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b)
        info[b] = potrf_one(n, A + (long long)b * sA, lda);
}

/* ------------------------------------------------------------------------ */
/* Triangular solves with the lower factor L (Sec. III-B "triangular ...     */
/* updates", "linear solves").                                              */
/*   forward : y_i = (b_i - sum_{k<i} l_ik y_k) / l_ii                       */
/*   backward: x_i = (y_i - sum_{k>i} l_ki x_k) / l_ii   (solves L^T x = y)   */
/* ------------------------------------------------------------------------ */
static void forward_lower(int n, const double *l, int lda, double *x, int unit)
{
    for (int i = 0; i < n; ++i) {
        double s = x[i];
        for (int k = 0; k < i; ++k)
            s -= l[k * lda + i] * x[k];
        x[i] = unit ? s : s / l[i * lda + i];
    }
}

static void backward_lower_transposed(int n, const double *l, int lda, double *x)
{
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k)
            s -= l[i * lda + k] * x[k];
        x[i] = s / l[i * lda + i];
    }
}

/* TRSM: left side, lower, no transpose, non-unit diagonal: L X = B, B <- X. */
void oracle_trsm_f64(int n, int nrhs, const double *L, int lda, long long sA,
                     double *B, int ldb, long long sB, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b)
        for (int c = 0; c < nrhs; ++c)
            forward_lower(n, L + (long long)b * sA, lda,
                          B + (long long)b * sB + (long long)c * ldb, 0);
}

/* POTRS: L L^T X = B with the factor from POTRF, B <- X. */
void oracle_potrs_f64(int n, int nrhs, const double *L, int lda, long long sA,
                      double *B, int ldb, long long sB, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b)
        for (int c = 0; c < nrhs; ++c) {
            const double *l = L + (long long)b * sA;
            double *x = B + (long long)b * sB + (long long)c * ldb;
            forward_lower(n, l, lda, x, 0);
            backward_lower_transposed(n, l, lda, x);
        }
}

/* POSV = POTRF then POTRS (Sec. III-A names glass::posv; Sec. IV-D POSV).
 * A <- L, B <- X; a matrix whose factorization fails keeps B unspecified. */
void oracle_posv_f64(int n, int nrhs, double *A, int lda, long long sA,
                     double *B, int ldb, long long sB, int *info, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        double *l = A + (long long)b * sA;
        info[b] = potrf_one(n, l, lda);
        if (info[b] != 0)
            continue;
        for (int c = 0; c < nrhs; ++c) {
            double *x = B + (long long)b * sB + (long long)c * ldb;
            forward_lower(n, l, lda, x, 0);
            backward_lower_transposed(n, l, lda, x);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* GETRF with partial pivoting, GETRS (Sec. III-B "factorizations, and       */
/* linear solves").  The step order is the unblocked right-looking textbook */
/* algorithm (LAPACK xGETF2):                                                */
/*   for j: p = argmax_{i>=j} |a_ij| (smallest i on ties); ipiv[j] = p;      */
/*          swap rows j and p in all n columns;                              */
/*          a_jj == 0 -> info = j+1 (first), column left unscaled (it is all */
/*          zero below the diagonal, so the update is a no-op);              */
/*          else a_ij /= a_jj (i>j); a_ik -= a_ij a_jk (i,k > j).            */
/* `gap` (optional, per problem) receives min over steps of                  */
/*  (|best| - |second best|) / |best| among the candidates, used by tests to */
/*  select inputs whose pivot choice is unambiguous.                         */
/* The routine is written once as a macro body so that the same steps can be */
/* run in FP64 and in FP32 (where a test needs the pivot decision taken in   */
/* the device's precision).                                                  */
/* ------------------------------------------------------------------------ */
#define DEFINE_GETRF_ONE(NAME, T, FABS)                                        \
static int NAME(int n, T *a, int lda, int *ipiv, double *gap)                 \
{                                                                             \
    int info = 0;                                                             \
    double g = 1.0;                                                           \
    for (int j = 0; j < n; ++j) {                                             \
        int p = j;                                                            \
        T best = FABS(a[j * lda + j]);                                        \
        T second = (T)0;                                                      \
        for (int i = j + 1; i < n; ++i) {                                     \
            T v = FABS(a[j * lda + i]);                                       \
            if (v > best) { second = best; best = v; p = i; }                 \
            else if (v > second) { second = v; }                              \
        }                                                                     \
        if (j + 1 < n && best > (T)0) {                                       \
            double r = ((double)best - (double)second) / (double)best;        \
            if (r < g) g = r;                                                 \
        }                                                                     \
        ipiv[j] = p;                                                          \
        if (p != j)                                                           \
            for (int c = 0; c < n; ++c) {                                     \
                T t = a[c * lda + j];                                         \
                a[c * lda + j] = a[c * lda + p];                              \
                a[c * lda + p] = t;                                           \
            }                                                                 \
        T piv = a[j * lda + j];                                               \
        if (piv == (T)0) {                                                    \
            if (info == 0) info = j + 1;                                      \
            continue;                                                         \
        }                                                                     \
        for (int i = j + 1; i < n; ++i)                                       \
            a[j * lda + i] = a[j * lda + i] / piv;                            \
        for (int k = j + 1; k < n; ++k)                                       \
            for (int i = j + 1; i < n; ++i)                                   \
                a[k * lda + i] -= a[j * lda + i] * a[k * lda + j];            \
    }                                                                         \
    if (gap) *gap = g;                                                        \
    return info;                                                              \
}

DEFINE_GETRF_ONE(getrf_one_f64, double, fabs)
DEFINE_GETRF_ONE(getrf_one_f32, float, fabsf)

void oracle_getrf_f64(int n, double *A, int lda, long long sA, int *ipiv,
                      int *info, double *gap, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b)
        info[b] = getrf_one_f64(n, A + (long long)b * sA, lda,
                                ipiv + (long long)b * n, gap ? gap + b : NULL);
}

/* The same steps in FP32 arithmetic (no FMA contraction: see the build
 * flags), for tests that need the pivot decision in single precision. */
void oracle_getrf_f32(int n, float *A, int lda, long long sA, int *ipiv,
                      int *info, double *gap, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b)
        info[b] = getrf_one_f32(n, A + (long long)b * sA, lda,
                                ipiv + (long long)b * n, gap ? gap + b : NULL);
}

/* GETRS: apply the row swaps to B in order j = 0..n-1, then forward solve
 * with the unit lower factor and backward solve with the upper factor. */
static void getrs_one(int n, const double *lu, int lda, const int *ipiv, double *x)
{
    for (int j = 0; j < n; ++j) {
        int p = ipiv[j];
        if (p != j) { double t = x[j]; x[j] = x[p]; x[p] = t; }
    }
    forward_lower(n, lu, lda, x, 1);
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int k = i + 1; k < n; ++k)
            s -= lu[k * lda + i] * x[k];
        x[i] = s / lu[i * lda + i];
    }
}

void oracle_getrs_f64(int n, int nrhs, const double *LU, int lda, long long sA,
                      const int *ipiv, double *B, int ldb, long long sB, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b)
        for (int c = 0; c < nrhs; ++c)
            getrs_one(n, LU + (long long)b * sA, lda, ipiv + (long long)b * n,
                      B + (long long)b * sB + (long long)c * ldb);
}

/* GETRF + GETRS in one call (the device library's fused getrf_getrs). */
void oracle_getrf_getrs_f64(int n, int nrhs, double *A, int lda, long long sA,
                            int *ipiv, double *B, int ldb, long long sB,
                            int *info, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        double *a = A + (long long)b * sA;
        int *pv = ipiv + (long long)b * n;
        info[b] = getrf_one_f64(n, a, lda, pv, NULL);
        if (info[b] != 0)
            continue;
        for (int c = 0; c < nrhs; ++c)
            getrs_one(n, a, lda, pv, B + (long long)b * sB + (long long)c * ldb);
    }
}

/* ------------------------------------------------------------------------ */
/* GEMM with operand transposes and scaling (Sec. III-B "BLAS L1-L3"; the     */
/* BLAS xGEMM definition):  C = alpha op(A) op(B) + beta C, op(X) = X or X^T, */
/* C m x n, op(A) m x k, op(B) k x n.  With beta == 0, C is not read.         */
/* ------------------------------------------------------------------------ */
void oracle_gemm_ex_f64(int ta, int tb, int m, int n, int k, double alpha,
                        const double *A, int lda, long long sA,
                        const double *B, int ldb, long long sB, double beta,
                        double *C, int ldc, long long sC, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *a = A + (long long)b * sA;
        const double *bb = B + (long long)b * sB;
        double *c = C + (long long)b * sC;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int l = 0; l < k; ++l) {
                    const double x = ta ? a[i * lda + l] : a[l * lda + i];
                    const double y = tb ? bb[l * ldb + j] : bb[j * ldb + l];
                    s += x * y;
                }
                c[j * ldc + i] = beta == 0.0 ? alpha * s : alpha * s + beta * c[j * ldc + i];
            }
    }
}

/* ------------------------------------------------------------------------ */
/* LQR feedback gain (Sec. III-B fused operations; Sec. IV-E):               */
/*   K = (R + B^T P B)^{-1} B^T P A                                          */
/* A nx x nx, B nx x nu, P nx x nx, R nu x nu, K nu x nx, each packed        */
/* column-major (leading dimension = rows) with its own batch stride.  The    */
/* steps follow the formula: PB = P B; S = R + B^T PB; PA = P A;              */
/* M = B^T PA; S = L L^T (POTRF, info); K = L^{-T} L^{-1} M (POTRS over the   */
/* nx columns of M).  K is unspecified where info != 0.                       */
/* ------------------------------------------------------------------------ */
void oracle_riccati_gain_f64(int nx, int nu, const double *A, long long sA,
                             const double *B, long long sB, const double *P, long long sP,
                             const double *R, long long sR, double *K, long long sK,
                             int *info, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *a = A + (long long)b * sA, *bm = B + (long long)b * sB;
        const double *p = P + (long long)b * sP, *r = R + (long long)b * sR;
        double *kk = K + (long long)b * sK;
        double *pb = (double *)malloc(sizeof(double) * (size_t)nx * nu);
        double *pa = (double *)malloc(sizeof(double) * (size_t)nx * nx);
        double *sm = (double *)malloc(sizeof(double) * (size_t)nu * nu);
        for (int i = 0; i < nx; ++i)          /* PB = P B */
            for (int j = 0; j < nu; ++j) {
                double s = 0.0;
                for (int l = 0; l < nx; ++l) s += p[l * nx + i] * bm[j * nx + l];
                pb[j * nx + i] = s;
            }
        for (int i = 0; i < nu; ++i)          /* S = R + B^T PB */
            for (int j = 0; j < nu; ++j) {
                double s = 0.0;
                for (int l = 0; l < nx; ++l) s += bm[i * nx + l] * pb[j * nx + l];
                sm[j * nu + i] = r[j * nu + i] + s;
            }
        for (int i = 0; i < nx; ++i)          /* PA = P A */
            for (int j = 0; j < nx; ++j) {
                double s = 0.0;
                for (int l = 0; l < nx; ++l) s += p[l * nx + i] * a[j * nx + l];
                pa[j * nx + i] = s;
            }
        for (int i = 0; i < nu; ++i)          /* M = B^T PA, into K */
            for (int j = 0; j < nx; ++j) {
                double s = 0.0;
                for (int l = 0; l < nx; ++l) s += bm[i * nx + l] * pa[j * nx + l];
                kk[j * nu + i] = s;
            }
        info[b] = potrf_one(nu, sm, nu);      /* S = L L^T */
        if (info[b] == 0)
            for (int c = 0; c < nx; ++c) {    /* K = S^{-1} M, column by column */
                forward_lower(nu, sm, nu, kk + (long long)c * nu, 0);
                backward_lower_transposed(nu, sm, nu, kk + (long long)c * nu);
            }
        free(pb);
        free(pa);
        free(sm);
    }
}

/* ------------------------------------------------------------------------ */
/* Rotation composition (Sec. III-B: SO(3) maps).  A chain of `chain` 3x3    */
/* column-major rotations R_0..R_{c-1} per problem, stored back to back      */
/* (9 values each), composes to R = R_0 R_1 ... R_{c-1}: R_{c-1} acts first. */
/* ------------------------------------------------------------------------ */
static void mat3_mul(const double *x, const double *y, double *z)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int l = 0; l < 3; ++l)
                s += x[l * 3 + i] * y[j * 3 + l];
            z[j * 3 + i] = s;
        }
}

void oracle_rot3_compose_f64(int chain, const double *Rs, long long sRs,
                             double *R, long long sR, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *in = Rs + (long long)b * sRs;
        double acc[9], tmp[9];
        memcpy(acc, in, sizeof acc);
        for (int c = 1; c < chain; ++c) {
            mat3_mul(acc, in + 9 * c, tmp);
            memcpy(acc, tmp, sizeof acc);
        }
        memcpy(R + (long long)b * sR, acc, sizeof acc);
    }
}

/* ------------------------------------------------------------------------ */
/* SE(3) apply (Sec. III-B: SE(3) maps).  A chain of `chain` 4x4 column-major*/
/* homogeneous transforms T_0..T_{c-1} per problem composes to               */
/* T = T_0 ... T_{c-1}; then q_i = R p_i + t with R = T[0:3,0:3],            */
/* t = T[0:3,3].  Points are 3 x npts column-major (x,y,z of point i at      */
/* 3i..3i+2).  The bottom row of each input transform is not read: it is     */
/* taken to be (0,0,0,1).                                                    */
/* ------------------------------------------------------------------------ */
void oracle_se3_apply_f64(int chain, const double *T, long long sT, int npts,
                          const double *P, long long sP, double *Q, long long sQ,
                          int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *tin = T + (long long)b * sT;
        double r[9], t[3];
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i)
                r[j * 3 + i] = tin[j * 4 + i];
        for (int i = 0; i < 3; ++i)
            t[i] = tin[12 + i];
        for (int c = 1; c < chain; ++c) {
            const double *tc = tin + 16 * c;
            double rc[9], nr[9], nt[3];
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < 3; ++i)
                    rc[j * 3 + i] = tc[j * 4 + i];
            /* [r t] [rc tc] = [r rc, r tc + t] */
            mat3_mul(r, rc, nr);
            for (int i = 0; i < 3; ++i) {
                double s = t[i];
                for (int l = 0; l < 3; ++l)
                    s += r[l * 3 + i] * tc[12 + l];
                nt[i] = s;
            }
            memcpy(r, nr, sizeof r);
            memcpy(t, nt, sizeof t);
        }
        const double *p = P + (long long)b * sP;
        double *q = Q + (long long)b * sQ;
        for (int k = 0; k < npts; ++k)
            for (int i = 0; i < 3; ++i) {
                double s = t[i];
                for (int l = 0; l < 3; ++l)
                    s += r[l * 3 + i] * p[3 * k + l];
                q[3 * k + i] = s;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Placement cost model: a 3-layer perceptron din -> h -> h -> dout with     */
/* ReLU, trained on log-latency with a masked mean-squared error and Adam.   */
/* The paper has no learned model (placements come from exhaustive offline  */
/* measurement, Sec. III-A); this is the plain definition of that network.   */
/* Weight layout (row-major, out x in):                                      */
/*   W1[h][din] b1[h] W2[h][h] b2[h] W3[dout][h] b3[dout], packed in order.  */
/* ------------------------------------------------------------------------ */
static void mlp_offsets(int din, int h, int dout, long long off[6])
{
    off[0] = 0;                        /* W1 */
    off[1] = off[0] + (long long)h * din;    /* b1 */
    off[2] = off[1] + h;               /* W2 */
    off[3] = off[2] + (long long)h * h;      /* b2 */
    off[4] = off[3] + h;               /* W3 */
    off[5] = off[4] + (long long)dout * h;   /* b3 */
}

long long oracle_mlp_nparams(int din, int h, int dout)
{
    long long off[6];
    mlp_offsets(din, h, dout, off);
    return off[5] + dout;
}

/* Forward for `rows` inputs X[rows][din] -> Y[rows][dout]. Optional H1, H2
 * ([rows][h]) receive the post-ReLU activations. */
void oracle_mlp_fwd_f64(int din, int h, int dout, const double *w, int rows,
                        const double *X, double *Y, double *H1, double *H2)
{
    long long off[6];
    mlp_offsets(din, h, dout, off);
    const double *W1 = w + off[0], *b1 = w + off[1], *W2 = w + off[2];
    const double *b2 = w + off[3], *W3 = w + off[4], *b3 = w + off[5];
    OMP_FOR
    for (int r = 0; r < rows; ++r) {
        double *h1 = (double *)malloc(sizeof(double) * h);
        double *h2 = (double *)malloc(sizeof(double) * h);
        const double *x = X + (long long)r * din;
        for (int o = 0; o < h; ++o) {
            double s = b1[o];
            for (int i = 0; i < din; ++i) s += W1[(long long)o * din + i] * x[i];
            h1[o] = s > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < h; ++o) {
            double s = b2[o];
            for (int i = 0; i < h; ++i) s += W2[(long long)o * h + i] * h1[i];
            h2[o] = s > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < dout; ++o) {
            double s = b3[o];
            for (int i = 0; i < h; ++i) s += W3[(long long)o * h + i] * h2[i];
            Y[(long long)r * dout + o] = s;
        }
        if (H1) memcpy(H1 + (long long)r * h, h1, sizeof(double) * h);
        if (H2) memcpy(H2 + (long long)r * h, h2, sizeof(double) * h);
        free(h1);
        free(h2);
    }
}

/* Masked MSE: loss = sum_{r,o} m_ro (y_ro - t_ro)^2 / max(1, sum m).
 * Returns the loss and writes dL/dw into grad (same layout as w). */
double oracle_mlp_loss_grad_f64(int din, int h, int dout, const double *w, int rows,
                                const double *X, const double *Tgt, const double *M,
                                double *grad)
{
    long long off[6];
    mlp_offsets(din, h, dout, off);
    long long np = off[5] + dout;
    const double *W2 = w + off[2], *W3 = w + off[4];
    double *H1 = (double *)malloc(sizeof(double) * (size_t)rows * h);
    double *H2 = (double *)malloc(sizeof(double) * (size_t)rows * h);
    double *Y = (double *)malloc(sizeof(double) * (size_t)rows * dout);
    oracle_mlp_fwd_f64(din, h, dout, w, rows, X, Y, H1, H2);
    double msum = 0.0;
    for (long long i = 0; i < (long long)rows * dout; ++i) msum += M[i];
    double denom = msum > 1.0 ? msum : 1.0;
    memset(grad, 0, sizeof(double) * (size_t)np);
    double loss = 0.0;
    double *dy = (double *)malloc(sizeof(double) * dout);
    double *d2 = (double *)malloc(sizeof(double) * h);
    double *d1 = (double *)malloc(sizeof(double) * h);
    for (int r = 0; r < rows; ++r) {
        const double *x = X + (long long)r * din;
        const double *h1 = H1 + (long long)r * h, *h2 = H2 + (long long)r * h;
        for (int o = 0; o < dout; ++o) {
            long long q = (long long)r * dout + o;
            double e = Y[q] - Tgt[q];
            loss += M[q] * e * e;
            dy[o] = 2.0 * M[q] * e / denom;
        }
        /* layer 3 */
        for (int o = 0; o < dout; ++o) {
            for (int i = 0; i < h; ++i)
                grad[off[4] + (long long)o * h + i] += dy[o] * h2[i];
            grad[off[5] + o] += dy[o];
        }
        for (int i = 0; i < h; ++i) {
            double s = 0.0;
            for (int o = 0; o < dout; ++o) s += W3[(long long)o * h + i] * dy[o];
            d2[i] = h2[i] > 0.0 ? s : 0.0;          /* ReLU'(z) = [z > 0] */
        }
        /* layer 2 */
        for (int o = 0; o < h; ++o) {
            for (int i = 0; i < h; ++i)
                grad[off[2] + (long long)o * h + i] += d2[o] * h1[i];
            grad[off[3] + o] += d2[o];
        }
        for (int i = 0; i < h; ++i) {
            double s = 0.0;
            for (int o = 0; o < h; ++o) s += W2[(long long)o * h + i] * d2[o];
            d1[i] = h1[i] > 0.0 ? s : 0.0;
        }
        /* layer 1 */
        for (int o = 0; o < h; ++o) {
            for (int i = 0; i < din; ++i)
                grad[off[0] + (long long)o * din + i] += d1[o] * x[i];
            grad[off[1] + o] += d1[o];
        }
    }
    free(dy); free(d2); free(d1);
    free(H1); free(H2); free(Y);
    return loss / denom;
}

/* One Adam step (Kingma & Ba 2015, Algorithm 1) at step count t >= 1:
 *   m = b1 m + (1-b1) g ; v = b2 v + (1-b2) g^2 ;
 *   w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)                   */
void oracle_adam_step_f64(long long np, double *w, const double *g, double *m,
                          double *v, int t, double lr, double b1, double b2,
                          double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (long long i = 0; i < np; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* ======================================================================== */
/* Robotics operations of the placement table of Sec. IV-E (Table II).      */
/* The paper fixes a convention per operation but does not print them; the  */
/* readings used here (and by the device library, by contract):             */
/*   quaternion q = (w, x, y, z), Hamilton product, unit norm;               */
/*   rotation vector d: angle |d| about d / |d|; Exp(d) = (cos |d|/2,         */
/*     sin(|d|/2) d / |d|); Log is its inverse on the w >= 0 hemisphere;     */
/*   quat_retract(q, d) = q * Exp(d)            (right perturbation);       */
/*   quat_error(q1, q2) = Log(conj(q1) * q2)    (so q2 = retract(q1, err));  */
/*   twist xi = (rho, phi): linear part first, angular second;              */
/*   se3_retract(T, xi) = T Exp(xi), T a 4x4 column-major homogeneous        */
/*     matrix, Exp(xi) = [Exp_SO3(phi), V(phi) rho; 0 1];                     */
/*   motion vectors (linear, angular); motion_cross(v, m) = v x m =          */
/*     (w x m_lin + v_lin x m_ang, w x m_ang) with w = v_ang;                */
/*   eig3: symmetric 3x3, eigenvalues ascending, eigenvector columns with    */
/*     their largest-magnitude component positive;                          */
/*   svd3: M = U diag(s) V^T, s descending and >= 0;                          */
/*   closest_rotation(M) = argmin_{R in SO(3)} |R - M|_F                      */
/*     = U diag(1, 1, det(U V^T)) V^T;                                      */
/*   argmax: first index of the largest value; softmax: exp(x - max) / sum.  */
/* ======================================================================== */
static void qmul(const double *a, const double *b, double *o)
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

static void qexp(const double *d, double *q)
{
    const double th = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double s = th > 0.0 ? sin(0.5 * th) / th : 0.5;
    q[0] = cos(0.5 * th);
    q[1] = s * d[0];
    q[2] = s * d[1];
    q[3] = s * d[2];
}

static void qlog(const double *qin, double *d)
{
    double q[4] = {qin[0], qin[1], qin[2], qin[3]};
    if (q[0] < 0.0)
        for (int i = 0; i < 4; ++i) q[i] = -q[i];
    const double nv = sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double f = nv > 0.0 ? 2.0 * atan2(nv, q[0]) / nv : 2.0 / q[0];
    for (int i = 0; i < 3; ++i) d[i] = f * q[i + 1];
}

void oracle_quat_retract_f64(const double *q, const double *d, double *out, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        double e[4];
        qexp(d + 3LL * b, e);
        qmul(q + 4LL * b, e, out + 4LL * b);
    }
}

void oracle_quat_error_f64(const double *q1, const double *q2, double *out, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *a = q1 + 4LL * b;
        const double c[4] = {a[0], -a[1], -a[2], -a[3]};
        double r[4];
        qmul(c, q2 + 4LL * b, r);
        qlog(r, out + 3LL * b);
    }
}

/* [p]x, column-major */
static void skew(const double *p, double *S)
{
    S[0] = 0.0;   S[3] = -p[2]; S[6] = p[1];
    S[1] = p[2];  S[4] = 0.0;   S[7] = -p[0];
    S[2] = -p[1]; S[5] = p[0];  S[8] = 0.0;
}

/* Exp of a twist: R = I + a S + b S^2, V = I + b S + c S^2, S = [phi]x,
 * a = sin t / t, b = (1 - cos t) / t^2 = 2 sin^2(t/2) / t^2,
 * c = (t - sin t) / t^3 (its Taylor series below t = 1e-2). */
static void se3_exp(const double *xi, double *T)
{
    const double *rho = xi, *phi = xi + 3;
    const double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], t = sqrt(t2);
    double a, bb, c;
    if (t > 0.0) {
        const double sh = sin(0.5 * t);
        a = sin(t) / t;
        bb = 2.0 * sh * sh / t2;
    } else {
        a = 1.0;
        bb = 0.5;
    }
    if (t < 1e-2)
        c = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0 - t2 * t2 * t2 / 362880.0;
    else
        c = (t - sin(t)) / (t2 * t);
    double S[9], S2[9], R[9], V[9];
    skew(phi, S);
    mat3_mul(S, S, S2);
    for (int k = 0; k < 9; ++k) {
        const double id = (k % 4 == 0) ? 1.0 : 0.0;
        R[k] = id + a * S[k] + bb * S2[k];
        V[k] = id + bb * S[k] + c * S2[k];
    }
    for (int k = 0; k < 16; ++k) T[k] = 0.0;
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) T[j * 4 + i] = R[j * 3 + i];
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += V[l * 3 + i] * rho[l];
        T[12 + i] = s;
    }
    T[15] = 1.0;
}

void oracle_se3_retract_f64(const double *T, const double *xi, double *out, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        double E[16];
        se3_exp(xi + 6LL * b, E);
        const double *t = T + 16LL * b;
        double *o = out + 16LL * b;
        for (int j = 0; j < 4; ++j)
            for (int i = 0; i < 4; ++i) {
                double s = 0.0;
                for (int l = 0; l < 4; ++l) s += (i == 3 ? (l == 3 ? 1.0 : 0.0) : t[l * 4 + i]) * E[j * 4 + l];
                o[j * 4 + i] = s;
            }
    }
}

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

void oracle_motion_cross_f64(const double *v, const double *m, double *out, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *vl = v + 6LL * b, *w = vl + 3, *ml = m + 6LL * b, *mw = ml + 3;
        double *o = out + 6LL * b, c1[3], c2[3];
        cross3(w, ml, c1);
        cross3(vl, mw, c2);
        for (int i = 0; i < 3; ++i) o[i] = c1[i] + c2[i];
        cross3(w, mw, o + 3);
    }
}

/* Cyclic Jacobi eigenvalue iteration on a symmetric 3x3 (col-major A),
 * to convergence in FP64; w ascending, V columns the eigenvectors. */
static void eig3_one(const double *Ain, double *w, double *Vout)
{
    double A[9], V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int k = 0; k < 9; ++k) A[k] = Ain[k];
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = A[3] * A[3] + A[6] * A[6] + A[7] * A[7];
        if (off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A[q * 3 + p];
                if (apq == 0.0) continue;
                const double app = A[p * 3 + p], aqq = A[q * 3 + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < 3; ++k) {
                    const double akp = A[p * 3 + k], akq = A[q * 3 + k];
                    A[p * 3 + k] = c * akp - s * akq;
                    A[q * 3 + k] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[k * 3 + p], aqk = A[k * 3 + q];
                    A[k * 3 + p] = c * apk - s * aqk;
                    A[k * 3 + q] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[p * 3 + k], vkq = V[q * 3 + k];
                    V[p * 3 + k] = c * vkp - s * vkq;
                    V[q * 3 + k] = s * vkp + c * vkq;
                }
            }
    }
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (A[idx[j] * 4] < A[idx[i] * 4]) { const int tmp = idx[i]; idx[i] = idx[j]; idx[j] = tmp; }
    for (int c = 0; c < 3; ++c) {
        w[c] = A[idx[c] * 4];
        int big = 0;
        for (int i = 1; i < 3; ++i)
            if (fabs(V[idx[c] * 3 + i]) > fabs(V[idx[c] * 3 + big])) big = i;
        const double sg = V[idx[c] * 3 + big] < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < 3; ++i) Vout[c * 3 + i] = sg * V[idx[c] * 3 + i];
    }
}

void oracle_eig3_f64(const double *A, double *w, double *V, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) eig3_one(A + 9LL * b, w + 3LL * b, V + 9LL * b);
}

/* SVD of a 3x3 through the eigen-decomposition of M^T M: V its
 * eigenvectors (descending), s = sqrt of the eigenvalues, U = M V / s with
 * the last column completed as u1 x u2 when s3 is zero. */
static void svd3_one(const double *M, double *U, double *s, double *V)
{
    double MtM[9], w[3], E[9];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += M[i * 3 + l] * M[j * 3 + l];
            MtM[j * 3 + i] = acc;
        }
    eig3_one(MtM, w, E);
    for (int c = 0; c < 3; ++c) {
        const int e = 2 - c;  /* descending */
        s[c] = sqrt(w[e] > 0.0 ? w[e] : 0.0);
        for (int i = 0; i < 3; ++i) V[c * 3 + i] = E[e * 3 + i];
    }
    for (int c = 0; c < 3; ++c) {
        double u[3];
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += M[l * 3 + i] * V[c * 3 + l];
            u[i] = acc;
        }
        for (int i = 0; i < 3; ++i) U[c * 3 + i] = s[c] > 0.0 ? u[i] / s[c] : 0.0;
    }
    if (!(s[2] > 0.0)) cross3(U, U + 3, U + 6);
}

void oracle_svd3_f64(const double *M, double *U, double *s, double *V, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) svd3_one(M + 9LL * b, U + 9LL * b, s + 3LL * b, V + 9LL * b);
}

void oracle_closest_rotation_f64(const double *M, double *R, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        double U[9], s[3], V[9], UVt[9];
        svd3_one(M + 9LL * b, U, s, V);
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) {
                double acc = 0.0;
                for (int l = 0; l < 3; ++l) acc += U[l * 3 + i] * V[l * 3 + j];
                UVt[j * 3 + i] = acc;
            }
        const double det = UVt[0] * (UVt[4] * UVt[8] - UVt[7] * UVt[5]) -
                           UVt[3] * (UVt[1] * UVt[8] - UVt[7] * UVt[2]) +
                           UVt[6] * (UVt[1] * UVt[5] - UVt[4] * UVt[2]);
        const double d[3] = {1.0, 1.0, det < 0.0 ? -1.0 : 1.0};
        double *r = R + 9LL * b;
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) {
                double acc = 0.0;
                for (int l = 0; l < 3; ++l) acc += U[l * 3 + i] * d[l] * V[l * 3 + j];
                r[j * 3 + i] = acc;
            }
    }
}

void oracle_argmax_f64(int n, const double *x, long long sx, int *idx, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *v = x + (long long)b * sx;
        int best = 0;
        for (int i = 1; i < n; ++i)
            if (v[i] > v[best]) best = i;
        idx[b] = best;
    }
}

void oracle_softmax_f64(int n, const double *x, long long sx, double *y, long long sy, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *v = x + (long long)b * sx;
        double *o = y + (long long)b * sy;
        double mx = v[0];
        for (int i = 1; i < n; ++i)
            if (v[i] > mx) mx = v[i];
        double s = 0.0;
        for (int i = 0; i < n; ++i) { o[i] = exp(v[i] - mx); s += o[i]; }
        for (int i = 0; i < n; ++i) o[i] /= s;
    }
}

/* ======================================================================== */
/* BLAS-1/2 and block-tridiagonal routines (Sec. III-B: "reductions, BLAS   */
/* L1-L3"; "block-tridiagonal matrix-vector products and direct ...        */
/* solvers commonly used in trajectory optimization").                     */
/* ======================================================================== */

/* dot: out[b] = sum_i x_i y_i over n entries (stride 1 within a problem). */
void oracle_dot_f64(int n, const double *x, long long sx, const double *y, long long sy,
                    double *out, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += x[(long long)b * sx + i] * y[(long long)b * sy + i];
        out[b] = s;
    }
}

/* gemv: y = alpha op(A) x + beta y, A m x n column-major (lda), op(A) = A
 * (trans 0, x has n entries, y m) or A^T (trans 1, x has m, y n); with
 * beta == 0, y is not read. */
void oracle_gemv_f64(int trans, int m, int n, double alpha, const double *A, int lda, long long sA,
                     const double *x, long long sx, double beta, double *y, long long sy, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const double *a = A + (long long)b * sA, *xb = x + (long long)b * sx;
        double *yb = y + (long long)b * sy;
        const int rows = trans ? n : m, inner = trans ? m : n;
        for (int i = 0; i < rows; ++i) {
            double s = 0.0;
            for (int l = 0; l < inner; ++l)
                s += (trans ? a[i * lda + l] : a[l * lda + i]) * xb[l];
            yb[i] = beta == 0.0 ? alpha * s : alpha * s + beta * yb[i];
        }
    }
}

/* The symmetric block-tridiagonal matrix T of N diagonal blocks D_i (nb x nb,
 * symmetric, all entries read) and N-1 sub-diagonal blocks O_i = T[i+1][i]
 * (the super-diagonal blocks are their transposes), assembled densely
 * (column-major, order N*nb). */
static void btd_assemble(int nb, int N, const double *D, const double *O, double *T)
{
    const int m = N * nb;
    for (int k = 0; k < m * m; ++k) T[k] = 0.0;
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < nb; ++c)
            for (int r = 0; r < nb; ++r) {
                T[(i * nb + c) * m + i * nb + r] = D[(long long)i * nb * nb + c * nb + r];
                if (i + 1 < N) {
                    const double o = O[(long long)i * nb * nb + c * nb + r];
                    T[(i * nb + c) * m + (i + 1) * nb + r] = o;      /* block (i+1, i) */
                    T[((i + 1) * nb + r) * m + i * nb + c] = o;      /* block (i, i+1) = O^T */
                }
            }
}

/* y = T x per problem (x, y of N*nb entries). */
void oracle_btd_matvec_f64(int nb, int N, const double *D, const double *O, const double *x,
                           double *y, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const int m = N * nb;
        double *T = (double *)malloc(sizeof(double) * (size_t)m * m);
        btd_assemble(nb, N, D + (long long)b * N * nb * nb, O + (long long)b * (N > 1 ? N - 1 : 0) * nb * nb, T);
        for (int r = 0; r < m; ++r) {
            double s = 0.0;
            for (int c = 0; c < m; ++c) s += T[c * m + r] * x[(long long)b * m + c];
            y[(long long)b * m + r] = s;
        }
        free(T);
    }
}

/* x = T^{-1} b for SPD T: the dense Cholesky solve of the assembled matrix
 * (POTRF + POTRS of this file).  info[b] is the dense POTRF info: the first
 * failing global column + 1. */
void oracle_btd_posv_f64(int nb, int N, const double *D, const double *O, double *bx, int *info,
                         int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const int m = N * nb;
        double *T = (double *)malloc(sizeof(double) * (size_t)m * m);
        btd_assemble(nb, N, D + (long long)b * N * nb * nb, O + (long long)b * (N > 1 ? N - 1 : 0) * nb * nb, T);
        info[b] = potrf_one(m, T, m);
        if (info[b] == 0) {
            forward_lower(m, T, m, bx + (long long)b * m, 0);
            backward_lower_transposed(m, T, m, bx + (long long)b * m);
        }
        free(T);
    }
}

/* Batched preconditioned conjugate gradient on the symmetric block-
 * tridiagonal T above: the iterative solver of the structured routines
 * (Sec. III-B names "direct and iterative solvers" for trajectory
 * optimization and fixes neither the method nor the preconditioner; the
 * reading here is the textbook PCG of Hestenes and Stiefel with the
 * block-Jacobi preconditioner M = blockdiag(D_0, ..., D_{N-1})):
 *   r = b - T x, z = M^{-1} r, p = z, rho = r'z, rho0 = rho;
 *   k = 0; while k < iters and rho > tol^2 rho0 (and rho > 0):
 *     q = T p; alpha = rho / p'q; x = x + alpha p; r = r - alpha q;
 *     z = M^{-1} r; rho_new = r'z; p = z + (rho_new / rho) p;
 *     rho = rho_new; k = k + 1.
 * M^{-1} v applies each D_i^{-1} by the dense Cholesky solve of D_i.  x holds
 * the initial guess on entry and the last iterate on return; iters_done[b]
 * is k, or -1 (x untouched) when some D_i is not positive definite, and the
 * loop also stops (k as reached) when p'Tp <= 0. */
void oracle_btd_pcg_f64(int nb, int N, const double *D, const double *O, const double *bv, double *x,
                        int iters, double tol, int *iters_done, int batch)
{
    OMP_FOR
    for (int b = 0; b < batch; ++b) {
        const int m = N * nb;
        const double *Db = D + (long long)b * N * nb * nb;
        const double *Ob = O + (long long)b * (N > 1 ? N - 1 : 0) * nb * nb;
        const double *bb = bv + (long long)b * m;
        double *xb = x + (long long)b * m;
        double *T = (double *)malloc(sizeof(double) * (size_t)m * m);
        double *L = (double *)malloc(sizeof(double) * (size_t)N * nb * nb);
        double *r = (double *)malloc(sizeof(double) * (size_t)m * 4);
        double *z = r + m, *p = z + m, *q = p + m;
        btd_assemble(nb, N, Db, Ob, T);
        int ok = 1;
        for (int i = 0; i < N && ok; ++i) {   /* Cholesky factors of the diagonal blocks */
            memcpy(L + (long long)i * nb * nb, Db + (long long)i * nb * nb, sizeof(double) * nb * nb);
            if (potrf_one(nb, L + (long long)i * nb * nb, nb) != 0) ok = 0;
        }
        if (!ok) {
            iters_done[b] = -1;
        } else {
            /* r = b - T x */
            for (int i = 0; i < m; ++i) {
                double s = 0.0;
                for (int c = 0; c < m; ++c) s += T[c * m + i] * xb[c];
                r[i] = bb[i] - s;
            }
            /* z = M^{-1} r */
            for (int i = 0; i < m; ++i) z[i] = r[i];
            for (int i = 0; i < N; ++i) {
                forward_lower(nb, L + (long long)i * nb * nb, nb, z + i * nb, 0);
                backward_lower_transposed(nb, L + (long long)i * nb * nb, nb, z + i * nb);
            }
            for (int i = 0; i < m; ++i) p[i] = z[i];
            double rho = 0.0;
            for (int i = 0; i < m; ++i) rho += r[i] * z[i];
            const double rho0 = rho;
            int k = 0;
            while (k < iters && rho > 0.0 && rho > tol * tol * rho0) {
                double pq = 0.0;
                for (int i = 0; i < m; ++i) {
                    double s = 0.0;
                    for (int c = 0; c < m; ++c) s += T[c * m + i] * p[c];
                    q[i] = s;
                    pq += p[i] * s;
                }
                if (!(pq > 0.0)) break;
                const double alpha = rho / pq;
                for (int i = 0; i < m; ++i) {
                    xb[i] += alpha * p[i];
                    r[i] -= alpha * q[i];
                }
                for (int i = 0; i < m; ++i) z[i] = r[i];
                for (int i = 0; i < N; ++i) {
                    forward_lower(nb, L + (long long)i * nb * nb, nb, z + i * nb, 0);
                    backward_lower_transposed(nb, L + (long long)i * nb * nb, nb, z + i * nb);
                }
                double rho_new = 0.0;
                for (int i = 0; i < m; ++i) rho_new += r[i] * z[i];
                const double beta = rho_new / rho;
                for (int i = 0; i < m; ++i) p[i] = z[i] + beta * p[i];
                rho = rho_new;
                ++k;
            }
            iters_done[b] = k;
        }
        free(r);
        free(L);
        free(T);
    }
}
