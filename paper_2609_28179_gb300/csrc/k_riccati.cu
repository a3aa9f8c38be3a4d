// k_riccati.cu -- batched GEMM with operand transposes and scaling
// (C = alpha op(A) op(B) + beta C), and the LQR feedback gain
// K = (R + B^T P B)^{-1} B^T P A fused into one kernel (Sec. III-B fused
// operations, Sec. IV-E): the team of one problem stages P, B and R in its
// shared memory, forms PB = P B, S = R + B^T PB and, with A staged over P,
// M = PB^T A (= B^T P A, P symmetric), factors S = L L^T and solves
// K = S^{-1} M, every intermediate on chip.  The unfused composition of the
// same steps (one library call per primitive, intermediates in global
// memory) is assembled in the C ABI; which of the two runs is a placement.
#include "common.cuh"

namespace glass {
namespace {

// Stage a rows x cols column-major operand (leading dimension ld) into
// shared memory with pitch p, 4-byte cp.async copies (any alignment).
template <int T>
__device__ __forceinline__ void stage_rect(float *dst, int p, const float *src, long long ld, int rows, int cols,
                                           int rank) {
    for (int e = rank; e < rows * cols; e += T) {
        const int c = e / rows, r = e - c * rows;
        cp_async4(dst + c * p + r, src + (long long)c * ld + r);
    }
}

// C(i,j) = alpha sum_l a(i,l) b(l,j) + beta C(i,j) (C not read when beta is
// 0) with a(i,l) = A[i*ai + l*al], b(l,j) = B[l*bl + j*bj] and
// C(i,j) = C[i + j*ldc]; the team's threads take the outputs in turn,
// consecutive threads consecutive rows.
template <int T>
__device__ __forceinline__ void team_gemm(int m, int n, int k, float alpha, const float *A, int ai, int al,
                                          const float *B, int bl, int bj, float beta, float *C, long long ldc,
                                          int rank) {
    for (int e = rank; e < m * n; e += T) {
        const int j = e / m, i = e - j * m;
        const float *a = A + i * ai;
        const float *b = B + j * bj;
        float s = 0.f;
        for (int l = 0; l < k; ++l) s = fmaf(a[l * al], b[l * bl], s);
        float *c = C + i + (long long)j * ldc;
        *c = beta == 0.f ? alpha * s : alpha * s + beta * *c;
    }
}

// Right-looking Cholesky of the lower triangle of S (order n, pitch p) by
// the team; dv[j] = 1 / l_jj.  Returns info (the same in every thread).
template <int T>
__device__ __forceinline__ int team_potrf(float *S, int p, int n, float *dv, int rank, int bar) {
    int info = 0;
    for (int j = 0; j < n; ++j) {
        const float d = S[j * p + j];
        if (!(d > 0.f) && info == 0) info = j + 1;
        const float l = sqrtf(d), r = 1.0f / l;
        team_sync<T>(bar);  // every thread has read the pivot
        if (rank == 0) {
            S[j * p + j] = l;
            dv[j] = r;
        }
        for (int i = j + 1 + rank; i < n; i += T) S[j * p + i] *= r;
        team_sync<T>(bar);
        const int m = n - j - 1;
        for (int e = rank; e < m * m; e += T) {
            const int c = j + 1 + e / m, i = j + 1 + e % m;
            if (i >= c) S[c * p + i] = fmaf(-S[j * p + i], S[j * p + c], S[c * p + i]);
        }
        team_sync<T>(bar);
    }
    return info;
}

template <int T, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_ex(int m, int n, int k, float alpha, Mat A, Mat B, float beta, Mat C,
                                                 int batch) {
    extern __shared__ float smem[];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const int b = blockIdx.x * (blockDim.x / T) + team;
    const int ra = TA ? k : m, ca = TA ? m : k, rb = TB ? n : k, cb = TB ? k : n;
    const int pa = ra | 1, pb = rb | 1;
    float *As = smem + team * (pa * ca + pb * cb);
    float *Bs = As + pa * ca;
    if (b >= batch) return;  // whole team
    stage_rect<T>(As, pa, A.p + (long long)b * A.s, A.ld, ra, ca, rank);
    stage_rect<T>(Bs, pb, B.p + (long long)b * B.s, B.ld, rb, cb, rank);
    cp_async_wait_all();
    team_sync<T>(1 + team);
    team_gemm<T>(m, n, k, alpha, As, TA ? pa : 1, TA ? 1 : pa, Bs, TB ? pb : 1, TB ? 1 : pb, beta,
                 C.p + (long long)b * C.s, C.ld, rank);
}

__host__ __device__ inline int riccati_floats_of(int nx, int nu) {
    const int px = nx | 1, pu = nu | 1;
    return px * nx + 2 * px * nu + pu * nu + pu * nx + nu;
}

template <int T>
__global__ void __launch_bounds__(256) k_riccati(int nx, int nu, const float *A, long long sA, const float *B,
                                                 long long sB, const float *P, long long sP, const float *R,
                                                 long long sR, float *K, long long sK, int *info, int batch) {
    extern __shared__ float smem[];
    const int team = threadIdx.x / T, rank = threadIdx.x % T, bar = 1 + team;
    const int b = blockIdx.x * (blockDim.x / T) + team;
    const int px = nx | 1, pu = nu | 1;  // odd pitches: column-strided team reads hit distinct banks
    float *W = smem + team * riccati_floats_of(nx, nu);  // P, then A
    float *Bm = W + px * nx, *PB = Bm + px * nu, *S = PB + px * nu, *M = S + pu * nu, *dv = M + pu * nx;
    if (b >= batch) return;  // whole team
    stage_rect<T>(W, px, P + (long long)b * sP, nx, nx, nx, rank);
    stage_rect<T>(Bm, px, B + (long long)b * sB, nx, nx, nu, rank);
    stage_rect<T>(S, pu, R + (long long)b * sR, nu, nu, nu, rank);
    cp_async_wait_all();
    team_sync<T>(bar);
    team_gemm<T>(nx, nu, nx, 1.f, W, 1, px, Bm, 1, px, 0.f, PB, px, rank);  // PB = P B
    team_sync<T>(bar);
    stage_rect<T>(W, px, A + (long long)b * sA, nx, nx, nx, rank);            // A over P, in flight ...
    team_gemm<T>(nu, nu, nx, 1.f, Bm, px, 1, PB, 1, px, 1.f, S, pu, rank);    // ... while S = R + B^T PB
    cp_async_wait_all();
    team_sync<T>(bar);
    team_gemm<T>(nu, nx, nx, 1.f, PB, px, 1, W, 1, px, 0.f, M, pu, rank);    // M = PB^T A
    const int inf = team_potrf<T>(S, pu, nu, dv, rank, bar);                 // S = L L^T (syncs order M too)
    for (int c = rank; c < nx; c += T) {                                       // K = L^{-T} L^{-1} M, a column each
        float *x = M + c * pu;
        for (int i = 0; i < nu; ++i) {
            const float xi = x[i] * dv[i];
            x[i] = xi;
            const float *l = S + i * pu;
            for (int r = i + 1; r < nu; ++r) x[r] = fmaf(-l[r], xi, x[r]);
        }
        for (int i = nu - 1; i >= 0; --i) {
            const float *l = S + i * pu;
            float s = x[i];
            for (int r = i + 1; r < nu; ++r) s = fmaf(-l[r], x[r], s);
            x[i] = s * dv[i];
        }
    }
    team_sync<T>(bar);
    float *k = K + (long long)b * sK;
    for (int e = rank; e < nu * nx; e += T) {
        const int c = e / nu, r = e - c * nu;
        k[(long long)c * nu + r] = M[c * pu + r];
    }
    if (rank == 0) info[b] = inf;
}

constexpr size_t kMaxSmem = 227 * 1024;

int team_of(Placement pl) { return pl.scope == SCOPE_WARP ? 32 : 128; }

size_t gemm_ex_floats(int ta, int tb, int m, int n, int k) {
    const int ra = ta ? k : m, ca = ta ? m : k, rb = tb ? n : k, cb = tb ? k : n;
    return (size_t)(ra | 1) * ca + (size_t)(rb | 1) * cb;
}

}  // namespace

size_t riccati_floats(int nx, int nu) { return (size_t)riccati_floats_of(nx, nu); }

bool feasible_gemm_ex(int ta, int tb, int m, int n, int k, Placement pl) {
    if (pl.scope != SCOPE_WARP && pl.scope != SCOPE_BLOCK) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (team_of(pl) * pl.pack > 256) return false;
    return gemm_ex_floats(ta, tb, m, n, k) * 4 * pl.pack <= kMaxSmem;
}

cudaError_t launch_gemm_ex(int ta, int tb, int m, int n, int k, float alpha, Mat A, Mat B, float beta, Mat C,
                           int batch, Placement pl, cudaStream_t st) {
    if (!feasible_gemm_ex(ta, tb, m, n, k, pl)) return cudaErrorInvalidConfiguration;
    const size_t smem = gemm_ex_floats(ta, tb, m, n, k) * 4 * pl.pack;
    const int grid = ceil_div(batch, pl.pack);
#define GL_GX(TT, X, Y)                                                                        \
    do {                                                                                       \
        auto kern = k_gemm_ex<TT, X, Y>;                                                       \
        cudaError_t e = prepare_kernel(reinterpret_cast<const void *>(kern), smem);            \
        if (e != cudaSuccess) return e;                                                        \
        kern<<<grid, TT * pl.pack, smem, st>>>(m, n, k, alpha, A, B, beta, C, batch);          \
        return cudaPeekAtLastError();                                                          \
    } while (0)
    if (team_of(pl) == 32) {
        if (ta && tb) GL_GX(32, true, true);
        if (ta) GL_GX(32, true, false);
        if (tb) GL_GX(32, false, true);
        GL_GX(32, false, false);
    }
    if (ta && tb) GL_GX(128, true, true);
    if (ta) GL_GX(128, true, false);
    if (tb) GL_GX(128, false, true);
    GL_GX(128, false, false);
#undef GL_GX
}

bool feasible_riccati(int nx, int nu, Placement pl) {
    if (nx < 1 || nx > 64 || nu < 1 || nu > 64) return false;
    if (pl.scope != SCOPE_WARP && pl.scope != SCOPE_BLOCK) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (team_of(pl) * pl.pack > 256) return false;
    return riccati_floats(nx, nu) * 4 * pl.pack <= kMaxSmem;
}

cudaError_t launch_riccati(int nx, int nu, const float *A, long long sA, const float *B, long long sB,
                           const float *P, long long sP, const float *R, long long sR, float *K, long long sK,
                           int *info, int batch, Placement pl, cudaStream_t st) {
    if (!feasible_riccati(nx, nu, pl)) return cudaErrorInvalidConfiguration;
    const size_t smem = riccati_floats(nx, nu) * 4 * pl.pack;
    const int grid = ceil_div(batch, pl.pack);
    const void *fn = team_of(pl) == 32 ? reinterpret_cast<const void *>(k_riccati<32>)
                                       : reinterpret_cast<const void *>(k_riccati<128>);
    cudaError_t e = prepare_kernel(fn, smem);
    if (e != cudaSuccess) return e;
    if (team_of(pl) == 32)
        k_riccati<32><<<grid, 32 * pl.pack, smem, st>>>(nx, nu, A, sA, B, sB, P, sP, R, sR, K, sK, info, batch);
    else
        k_riccati<128><<<grid, 128 * pl.pack, smem, st>>>(nx, nu, A, sA, B, sB, P, sP, R, sR, K, sK, info, batch);
    return cudaPeekAtLastError();
}

}  // namespace glass
