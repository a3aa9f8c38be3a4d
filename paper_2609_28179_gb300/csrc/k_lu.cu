// k_lu.cu -- batched getrf + getrs (partial pivoting) at thread, warp and
// block scope.  Thread scope stages 32*pack problems through shared memory;
// warp scope loads rows straight into registers up to order 16 -- two
// problems per warp, one per half -- and runs the blocked tensor-core
// factorization (dev_lu_tc.cuh) on the problem in shared memory above that;
// block scope is a 64-thread row team (dev_rows.cuh), one row per thread,
// up to order 32 and a two-warp team on the blocked tensor-core
// factorization (dev_lu_tc2.cuh) above.
#include "dev_lu.cuh"
#include "dev_lu_tc.cuh"
#include "dev_lu_tc2.cuh"
#include "dev_rows.cuh"

namespace glass {
namespace {

template <int NMAX, bool EXACT>
__global__ void __launch_bounds__(256) k_lu_thread(int n_rt, int nrhs, Mat A, int *ipiv, Mat B, int *info,
                                                   int batch) {
    extern __shared__ float smem[];
    const int n = EXACT ? NMAX : n_rt;
    const int G = blockDim.x;
    const int b0 = blockIdx.x * G;
    const int cnt = min(G, batch - b0);
    const int t = threadIdx.x;
    const bool staged = A.layout == GLASS_LAYOUT_COLMAJOR;
    const int SA = odd_stride(n * n);
    const int SB = nrhs > 0 ? odd_stride(n * nrhs) : 0;
    float *sa = smem;
    float *sb = smem + G * SA;
    if (staged) {
        stage_in(sa, SA, A, b0, cnt);
        if (nrhs > 0) stage_in(sb, SB, B, b0, cnt);
        __syncthreads();
    }
    if (t < cnt) {
        const int b = b0 + t;
        float *pa = sa + t * SA;
        float a[NMAX][NMAX];
        int piv[NMAX];
        float rinv[NMAX];
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                a[i][j] = (i < n && j < n) ? (staged ? pa[j * n + i] : A.get(b, i, j)) : 0.f;
        info[b] = thread::getrf<NMAX, EXACT>(a, piv, rinv, n);
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
            if (j < n) ipiv[(long long)b * n + j] = piv[j];
        float *pb = sb + t * SB;
        float *wb = opaque(pb);
        for (int c = 0; c < nrhs; ++c) {
            float x[NMAX];
#pragma unroll
            for (int i = 0; i < NMAX; ++i) x[i] = (i < n) ? (staged ? pb[c * n + i] : B.get(b, i, c)) : 0.f;
            thread::getrs<NMAX, EXACT>(a, piv, rinv, x, n);
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                if (i < n) {
                    if (staged) wb[c * n + i] = x[i];
                    else B.set(b, i, c, x[i]);
                }
        }
        float *wa = opaque(pa);
#pragma unroll
        for (int j = 0; j < NMAX; ++j)
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                if (i < n && j < n) {
                    if (staged) wa[j * n + i] = a[i][j];
                    else A.set(b, i, j, a[i][j]);
                }
    }
    if (staged) {
        __syncthreads();
        stage_out(sa, SA, A, b0, cnt);
        if (nrhs > 0) stage_out(sb, SB, B, b0, cnt);
    }
}

// Warp scope, orders up to 16: two problems per warp, one per half (row r in
// lane 16 h + r); half-warp primitive of dev_lu.cuh.  A half without a
// problem (odd batch) runs on zeros and stores nothing: the shuffles need
// the whole warp.
template <int NMAX>
__global__ void __launch_bounds__(256) k_lu_half(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch) {
    extern __shared__ int hsmem[];
    const int lane = threadIdx.x & 31, r = lane & 15, h = lane >> 4, w = threadIdx.x >> 5;
    int *sm = hsmem + (2 * w + h) * 2 * NMAX;
    const long long pair = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    if (2 * pair >= batch) return;  // whole warp
    const long long b = 2 * pair + h;
    const bool live = b < batch;
    float a[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) a[k] = (live && k < n && r < n) ? A.cget(b, r, k) : 0.f;
    int pos;
    const int inf = half::getrf<NMAX>(a, pos, sm, live ? ipiv + b * n : nullptr, n);
    if (live && r == 0) info[b] = inf;
#pragma unroll 1
    for (int c = 0; c < nrhs; ++c) {
        float x = (live && r < n) ? B.cget(b, r, c) : 0.f;
        half::getrs<NMAX>(a, pos, sm, x, n);
        if (live && r < n) B.cset(b, pos, c, x);
    }
    if (live && r < n) {
        float *wa = opaque(A.p + b * A.s);
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < n) wa[(long long)k * A.ld + pos] = a[k];
    }
}

// Warp scope, orders 33..64: blocked LU with tensor-core trailing updates on
// the problem held in the warp's shared memory (dev_lu_tc.cuh); per warp
// A (NMAX x LD), 1/u_jj, the interchanges and the original row of each
// logical row (the solve gathers b through it).
template <int NMAX>
constexpr int lu_tc_floats() {
    return NMAX * tclu::Shape<NMAX>::LD + 3 * NMAX;
}

// Orders 17..32 cap the registers at 80 (three blocks of 256 threads), so 24
// warps fit on an SM instead of 18 (n = 24 / 32 at batch 16384: 84 -> 71 and
// 97 -> 82 us); order 64 is bound by shared memory (12 warps) either way.
template <int NMAX>
__global__ void __launch_bounds__(256, NMAX == 32 ? 3 : 1) k_lu_tc(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch) {
    constexpr int LD = tclu::Shape<NMAX>::LD;
    constexpr int R = tclu::Shape<NMAX>::R;
    extern __shared__ __align__(16) float smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *As = smem + w * lu_tc_floats<NMAX>();
    float *dv = As + NMAX * LD;
    int *ps = reinterpret_cast<int *>(dv + NMAX);
    int *prow = ps + NMAX;
    const int b = blockIdx.x * (blockDim.x >> 5) + w;
    if (b >= batch) return;  // whole warp
#pragma unroll
    for (int q = 0; q < R; ++q) prow[lane + 32 * q] = lane + 32 * q;
    tcwarp::stage_async<NMAX, false, LD>(As, A.p + (long long)b * A.s, A.ld, n);
    tcwarp::wait_first();  // the first panel starts while columns 16.. arrive
    const int inf = tclu::getrf<NMAX>(As, n, prow, ps, dv);
    if (lane == 0) info[b] = inf;
    int *gp = ipiv + (long long)b * n;
    for (int j = lane; j < n; j += 32) gp[j] = ps[j];
    for (int c = 0; c < nrhs; ++c) {
        float x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            x[q] = (i < n) ? B.cget(b, prow[i], c) : 0.f;
        }
        tclu::getrs<NMAX>(As, dv, x, n);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = lane + 32 * q;
            if (i < n) B.cset(b, i, c, x[q]);
        }
    }
    tcwarp::unstage<NMAX, false, LD>(A.p + (long long)b * A.s, A.ld, As, n);
}

// Block scope, orders 33..64: the blocked tensor-core LU run by a team of
// two warps per problem (dev_lu_tc2.cuh); afterwards warp 0 solves and
// warp 1 writes the factor, the interchanges and info back.
__global__ void __launch_bounds__(256) k_lu_tc2(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch) {
    constexpr int NMAX = tclu2::NMAX, LD = tclu2::LD;
    extern __shared__ __align__(16) float smem[];
    const int team = threadIdx.x / tclu2::T, rank = threadIdx.x % tclu2::T;
    const int b = blockIdx.x * (blockDim.x / tclu2::T) + team;
    const int bid = 1 + team;
    float *As = smem + team * tclu2::floats();
    float *dv = As + NMAX * LD;
    int *ps = reinterpret_cast<int *>(dv + NMAX);
    int *prow = ps + NMAX;
    float *xch = reinterpret_cast<float *>(prow + NMAX);
    if (b >= batch) return;  // the whole team leaves together
    prow[rank] = rank;
    tclu2::stage(As, A.p + (long long)b * A.s, A.ld, n, rank, bid);  // ends with a team barrier
    const int inf = tclu2::getrf(As, n, prow, ps, dv, xch, rank, bid);
    const int lane = rank & 31;
    if (rank < 32) {
        for (int c = 0; c < nrhs; ++c) {
            float x[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i = lane + 32 * q;
                x[q] = (i < n) ? B.cget(b, prow[i], c) : 0.f;
            }
            tclu::getrs<NMAX>(As, dv, x, n);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i = lane + 32 * q;
                if (i < n) B.cset(b, i, c, x[q]);
            }
        }
    } else {
        if (lane == 0) info[b] = inf;
        int *gp = ipiv + (long long)b * n;
        for (int j = lane; j < n; j += 32) gp[j] = ps[j];
        tcwarp::unstage<NMAX, false, LD>(A.p + (long long)b * A.s, A.ld, As, n);
    }
}

constexpr int kRS = 4;

template <int NMAX>
constexpr int lu_team_floats() {
    return ((rows::Scratch<NMAX, kRS>::floats + 3) / 4) * 4;
}

template <int NMAX>
__global__ void __launch_bounds__(256) k_lu_rows(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch) {
    extern __shared__ __align__(16) float smem[];
    const int team = threadIdx.x / rows::T, i = threadIdx.x % rows::T;
    const int b = blockIdx.x * (blockDim.x / rows::T) + team;
    const int bid = 1 + team;
    rows::Scratch<NMAX, kRS> s(smem + team * lu_team_floats<NMAX>());
    if (b >= batch) return;
    float a[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) a[k] = (k < n && i < n) ? A.cget(b, i, k) : 0.f;
    int pos;
    bool done;
    const int inf = rows::getrf<NMAX, kRS>(a, pos, done, n, i, s, ipiv + (long long)b * n, bid);
    if (i == 0) info[b] = inf;
    for (int c0 = 0; c0 < nrhs; c0 += kRS) {
        float x[kRS];
#pragma unroll
        for (int c = 0; c < kRS; ++c) x[c] = (i < n && c0 + c < nrhs) ? B.cget(b, i, c0 + c) : 0.f;
        rows::getrs<NMAX, kRS>(a, pos, x, n, i, s, bid);
        if (i < n)
#pragma unroll
            for (int c = 0; c < kRS; ++c)
                if (c0 + c < nrhs) B.cset(b, pos, c0 + c, x[c]);
    }
    if (i < n)
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < n) A.cset(b, pos, k, a[k]);
}

template <typename K>
cudaError_t go(K kern, int grid, int threads, size_t smem, cudaStream_t st, int n, int nrhs, const Mat &A, int *ipiv,
               const Mat &B, int *info, int batch) {
    {
        cudaError_t e = prepare(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, threads, smem, st>>>(n, nrhs, A, ipiv, B, info, batch);
    return cudaPeekAtLastError();
}

constexpr size_t kMaxSmem = 227 * 1024;

size_t smem_lu(int n, int nrhs, Placement pl) {
    switch (pl.scope) {
        case SCOPE_THREAD: return (size_t)32 * pl.pack * (odd_stride(n * n) + (nrhs > 0 ? odd_stride(n * nrhs) : 0)) * 4;
        case SCOPE_WARP:
            return n > 32   ? (size_t)pl.pack * lu_tc_floats<64>() * 4
                   : n > 16 ? (size_t)pl.pack * lu_tc_floats<32>() * 4
                            : (size_t)pl.pack * 4 * 16 * 4;
        default: {
            if (n > 32) return (size_t)pl.pack * tclu2::floats() * 4;
            const int N = n <= 8 ? 8 : n <= 16 ? 16 : 32;
            const int f = N == 8 ? lu_team_floats<8>() : N == 16 ? lu_team_floats<16>() : lu_team_floats<32>();
            return (size_t)pl.pack * f * 4;
        }
    }
}

}  // namespace

bool feasible_lu(int n, int nrhs, Placement pl) {
    if (n < 1 || n > 64 || nrhs < 0) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (pl.scope == SCOPE_THREAD && n > 12) return false;
    if (pl.scope == SCOPE_BLOCK && rows::T * pl.pack > 256) return false;
    return smem_lu(n, nrhs, pl) <= kMaxSmem;
}

cudaError_t launch_getrf_getrs(int n, int nrhs, Mat A, int *ipiv, Mat B, int *info, int batch, Placement pl,
                               cudaStream_t st) {
    if (!feasible_lu(n, nrhs, pl)) return cudaErrorInvalidConfiguration;
    const size_t smem = smem_lu(n, nrhs, pl);
    if (pl.scope == SCOPE_THREAD) {
        const int G = 32 * pl.pack;
        const int grid = ceil_div(batch, G);
        const size_t sm = A.layout == GLASS_LAYOUT_COLMAJOR ? smem : 0;
#define GL_T(N, EX) go(k_lu_thread<N, EX>, grid, G, sm, st, n, nrhs, A, ipiv, B, info, batch)
        switch (n) {
            case 3: return GL_T(3, true);
            case 6: return GL_T(6, true);
            case 7: return GL_T(7, true);
            case 12: return GL_T(12, true);
            default: break;
        }
        if (n <= 2) return GL_T(2, false);
        if (n <= 4) return GL_T(4, false);
        if (n <= 8) return GL_T(8, false);
        return GL_T(12, false);
#undef GL_T
    }
    const int grid = ceil_div(batch, pl.pack);
    if (pl.scope == SCOPE_WARP) {
        const int th = 32 * pl.pack;
        if (n > 32) return go(k_lu_tc<64>, grid, th, smem, st, n, nrhs, A, ipiv, B, info, batch);
        if (n > 16) return go(k_lu_tc<32>, grid, th, smem, st, n, nrhs, A, ipiv, B, info, batch);
        // orders up to 16: two problems per warp (half-warp primitive)
        const int N = n <= 8 ? 8 : 16;
        const size_t sw = (size_t)pl.pack * 4 * N * 4;
        const int g2 = ceil_div(batch, 2 * pl.pack);
        if (N == 8) return go(k_lu_half<8>, g2, th, sw, st, n, nrhs, A, ipiv, B, info, batch);
        return go(k_lu_half<16>, g2, th, sw, st, n, nrhs, A, ipiv, B, info, batch);
    }
    const int th = rows::T * pl.pack;
    if (n > 32) return go(k_lu_tc2, grid, tclu2::T * pl.pack, smem, st, n, nrhs, A, ipiv, B, info, batch);
    if (n <= 8) return go(k_lu_rows<8>, grid, th, smem, st, n, nrhs, A, ipiv, B, info, batch);
    if (n <= 16) return go(k_lu_rows<16>, grid, th, smem, st, n, nrhs, A, ipiv, B, info, batch);
    return go(k_lu_rows<32>, grid, th, smem, st, n, nrhs, A, ipiv, B, info, batch);
}

}  // namespace glass
