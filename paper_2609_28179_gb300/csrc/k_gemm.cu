// k_gemm.cu -- batched SIMT GEMM C = A B (FP32) at thread, warp and block
// scope (Sec. III-B BLAS-3; the GEMM family of Sec. IV-D).
//
// Thread scope: one product per thread; A in registers, B and C streamed a
// column at a time through the CTA's staging buffers.
// Warp / block scope: a team of T threads per product.  A (column-major)
// and B (transposed, so that a row of B is contiguous) are staged into the
// team's shared memory with coalesced loads; each thread accumulates a
// TM x TN register tile of C from 16-byte shared-memory fragments (the
// warp's lanes share rows and columns, so fragments are mostly broadcasts);
// C goes back through shared memory for fully coalesced streaming stores.
// Block scope, pack 1, order 64 on packed 16-byte aligned operands goes to
// the fifth-generation tensor cores instead (3xTF32, k_gemm_tc.cu).
#include "common.cuh"

namespace glass {
namespace {

// ------------------------------------------------------------ thread scope
template <int NMAX, bool EXACT>
__global__ void __launch_bounds__(256) k_gemm_thread(int m_rt, int n_rt, int k_rt, Mat A, Mat B, Mat C, int batch) {
    extern __shared__ float smem[];
    const int m = EXACT ? NMAX : m_rt, n = EXACT ? NMAX : n_rt, k = EXACT ? NMAX : k_rt;
    const int G = blockDim.x;
    const int b0 = blockIdx.x * G;
    const int cnt = min(G, batch - b0);
    const int t = threadIdx.x;
    const bool staged = A.layout == GLASS_LAYOUT_COLMAJOR;
    const int SA = odd_stride(m * k), SB = odd_stride(k * n), SC = odd_stride(m * n);
    float *sa = smem, *sb = sa + G * SA, *sc = sb + G * SB;
    if (staged) {
        stage_in(sa, SA, A, b0, cnt);
        stage_in(sb, SB, B, b0, cnt);
        __syncthreads();
    }
    if (t < cnt) {
        const int b = b0 + t;
        float a[NMAX][NMAX];
#pragma unroll
        for (int l = 0; l < NMAX; ++l)
#pragma unroll
            for (int i = 0; i < NMAX; ++i)
                a[i][l] = (i < m && l < k) ? (staged ? sa[t * SA + l * m + i] : A.get(b, i, l)) : 0.f;
        for (int j = 0; j < n; ++j) {
            float bc[NMAX];
#pragma unroll
            for (int l = 0; l < NMAX; ++l) bc[l] = (l < k) ? (staged ? sb[t * SB + j * k + l] : B.get(b, l, j)) : 0.f;
#pragma unroll
            for (int i = 0; i < NMAX; ++i) {
                if (i < m) {
                    float c = 0.f;
#pragma unroll
                    for (int l = 0; l < NMAX; ++l)
                        if (l < k) c = fmaf(a[i][l], bc[l], c);
                    if (staged) sc[t * SC + j * m + i] = c;
                    else C.set(b, i, j, c);
                }
            }
        }
    }
    if (staged) {
        __syncthreads();
        stage_out(sc, SC, C, b0, cnt);
    }
}

// ------------------------------------------------------ warp / block scope
// Thread tile of a team of T threads on an NMAX x NMAX product.
template <int NMAX, int T>
struct Tile {
    static constexpr int area = NMAX * NMAX / T;  // C elements per thread
    static constexpr int TM = area >= 64 ? 8 : (area >= 16 ? 4 : (area >= 4 ? 2 : 1));
    static constexpr int TN = area / TM;
    static constexpr int RG = NMAX / TM;  // row groups
    static constexpr int CG = NMAX / TN;  // column groups
    static_assert(RG * CG == T, "tile does not cover the product");
    static constexpr int LD = NMAX + 4;  // smem leading dimension (16-byte rows)
    static constexpr int per = 2 * NMAX * LD;  // floats of staging per team
};

template <int N>
__device__ __forceinline__ void load_frag(float (&r)[N], const float *p) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int u = 0; u < N; u += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p + u);
            r[u] = v.x; r[u + 1] = v.y; r[u + 2] = v.z; r[u + 3] = v.w;
        }
    } else if constexpr (N == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        r[0] = v.x; r[1] = v.y;
    } else {
#pragma unroll
        for (int u = 0; u < N; ++u) r[u] = p[u];
    }
}

template <int NMAX, int T>
__global__ void __launch_bounds__(256) k_gemm_team(int m, int n, int k, Mat A, Mat B, Mat C, int batch) {
    using TL = Tile<NMAX, T>;
    extern __shared__ __align__(16) float smem[];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const int P = blockDim.x / T;
    const int b = blockIdx.x * P + team;
    const int bar = 1 + team;
    float *As = smem + team * TL::per;        // As[l*LD + i] = A(i, l)
    float *Bt = As + NMAX * TL::LD;           // Bt[l*LD + j] = B(l, j)
    if (b >= batch) return;
    // stage (zero padding outside m x k / k x n)
    const bool pk = A.packed() && B.packed();
    for (int e = rank; e < NMAX * NMAX; e += T) {
        const int l = e / NMAX, i = e - l * NMAX;
        float v = 0.f;
        if (i < m && l < k) v = pk ? __ldcs(A.p + (long long)b * A.s + l * m + i) : A.get(b, i, l);
        As[l * TL::LD + i] = v;
    }
    for (int e = rank; e < NMAX * NMAX; e += T) {
        const int j = e / NMAX, l = e - j * NMAX;
        float v = 0.f;
        if (l < k && j < n) v = pk ? __ldcs(B.p + (long long)b * B.s + j * k + l) : B.get(b, l, j);
        Bt[l * TL::LD + j] = v;
    }
    team_sync<T>(bar);
    const int rg = rank / TL::CG, cg = rank % TL::CG;
    const int i0 = rg * TL::TM, j0 = cg * TL::TN;
    float acc[TL::TM][TL::TN];
#pragma unroll
    for (int r = 0; r < TL::TM; ++r)
#pragma unroll
        for (int c = 0; c < TL::TN; ++c) acc[r][c] = 0.f;
#pragma unroll 4
    for (int l = 0; l < NMAX; ++l) {
        float af[TL::TM], bf[TL::TN];
        load_frag<TL::TM>(af, As + l * TL::LD + i0);
        load_frag<TL::TN>(bf, Bt + l * TL::LD + j0);
#pragma unroll
        for (int r = 0; r < TL::TM; ++r)
#pragma unroll
            for (int c = 0; c < TL::TN; ++c) acc[r][c] = fmaf(af[r], bf[c], acc[r][c]);
    }
    team_sync<T>(bar);
    // C tile -> shared (column-major, ld = m) -> coalesced stores
    float *Cs = As;
#pragma unroll
    for (int c = 0; c < TL::TN; ++c)
#pragma unroll
        for (int r = 0; r < TL::TM; ++r) {
            const int i = i0 + r, j = j0 + c;
            if (i < m && j < n) Cs[j * m + i] = acc[r][c];
        }
    team_sync<T>(bar);
    if (C.packed()) {
        float *g = C.p + (long long)b * C.s;
        const int tot = m * n;
        if (((reinterpret_cast<uintptr_t>(g) & 15) == 0) && (tot & 3) == 0) {
            for (int v = rank; v < (tot >> 2); v += T)
                __stcs(reinterpret_cast<float4 *>(g) + v, *reinterpret_cast<const float4 *>(Cs + 4 * v));
        } else {
            for (int e = rank; e < tot; e += T) __stcs(g + e, Cs[e]);
        }
    } else {
        for (int e = rank; e < m * n; e += T) {
            const int j = e / m, i = e - j * m;
            C.set(b, i, j, Cs[e]);
        }
    }
}

// Block scope, n a multiple of 4, packed 16-byte aligned operands: A and B
// staged column-major (pitch NMAX + 4) with cp.async 16-byte copies; the
// inner loop takes four k at a time so each B fragment is one 16-byte read
// of a column of B.  Lanes are laid out row-group fastest: the 8 lanes of
// a quarter-warp share their B columns (broadcast) and read 8 consecutive
// 16-byte A fragments (no bank conflict).  C goes back through shared
// memory for coalesced 16-byte stores.
template <int NMAX, int T>
__global__ void __launch_bounds__(T) k_gemm_async(int n, Mat A, Mat B, Mat C, int batch) {
    constexpr int TM = 4, TN = 4;
    constexpr int RG = NMAX / TM, CG = NMAX / TN;
    static_assert(RG * CG == T, "tile does not cover the product");
    constexpr int LD = NMAX + 4;
    extern __shared__ __align__(16) float smem[];
    float *As = smem, *Bs = smem + NMAX * LD;
    const int b = blockIdx.x;
    const int rank = threadIdx.x;
    const int q4 = n >> 2;
    const float *ga = A.p + (long long)b * A.s, *gb = B.p + (long long)b * B.s;
    for (int e = rank; e < n * q4; e += T) {
        const int c = e / q4, q = e - c * q4;
        cp_async16(As + c * LD + 4 * q, ga + c * n + 4 * q);
        cp_async16(Bs + c * LD + 4 * q, gb + c * n + 4 * q);
    }
    // zero padding when n < NMAX
    for (int e = rank; e < NMAX * NMAX; e += T) {
        const int c = e / NMAX, r = e - c * NMAX;
        if (r >= n || c >= n) { As[c * LD + r] = 0.f; Bs[c * LD + r] = 0.f; }
    }
    cp_async_wait_all();
    __syncthreads();
    const int rg = rank % RG, cg = rank / RG;
    const int i0 = rg * TM, j0 = cg * TN;
    float acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = 0.f;
#pragma unroll 2
    for (int l = 0; l < NMAX; l += 4) {
        float bq[TN][4];
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const float4 v = *reinterpret_cast<const float4 *>(Bs + (j0 + c) * LD + l);
            bq[c][0] = v.x; bq[c][1] = v.y; bq[c][2] = v.z; bq[c][3] = v.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 a = *reinterpret_cast<const float4 *>(As + (l + u) * LD + i0);
            const float af[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[r][c] = fmaf(af[r], bq[c][u], acc[r][c]);
        }
    }
    __syncthreads();
    float *Cs = As;
#pragma unroll
    for (int c = 0; c < TN; ++c)
        *reinterpret_cast<float4 *>(Cs + (j0 + c) * LD + i0) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
    __syncthreads();
    float *gc = C.p + (long long)b * C.s;
    for (int e = rank; e < n * q4; e += T) {
        const int c = e / q4, q = e - c * q4;
        __stcs(reinterpret_cast<float4 *>(gc + c * n + 4 * q), *reinterpret_cast<const float4 *>(Cs + c * LD + 4 * q));
    }
}

// Block scope at order 64: the same staging with a 64-thread team, each
// thread an 8 x 8 tile made of two 4-row and two 4-column halves 32 apart
// (rows 4g..4g+3 and 32+4g..32+4g+3), so the 8 lanes of a quarter-warp
// read 8 distinct 16-byte bank groups of A and share B (broadcast): per
// four k, 16 16-byte reads feed 256 fused multiply-adds.
template <int NMAX>
__global__ void __launch_bounds__(64) k_gemm_async8(int n, Mat A, Mat B, Mat C, int batch) {
    static_assert(NMAX == 64, "the 8x8 tiling covers a 64x64 product with 64 threads");
    constexpr int LD = NMAX + 4;
    extern __shared__ __align__(16) float smem[];
    float *As = smem, *Bs = smem + NMAX * LD;
    const int b = blockIdx.x;
    const int rank = threadIdx.x;
    const int q4 = n >> 2;
    const float *ga = A.p + (long long)b * A.s, *gb = B.p + (long long)b * B.s;
    for (int e = rank; e < n * q4; e += 64) {
        const int c = e / q4, q = e - c * q4;
        cp_async16(As + c * LD + 4 * q, ga + c * n + 4 * q);
        cp_async16(Bs + c * LD + 4 * q, gb + c * n + 4 * q);
    }
    for (int e = rank; e < NMAX * NMAX; e += 64) {  // zero padding when n < NMAX
        const int c = e / NMAX, r = e - c * NMAX;
        if (r >= n || c >= n) { As[c * LD + r] = 0.f; Bs[c * LD + r] = 0.f; }
    }
    cp_async_wait_all();
    __syncthreads();
    const int rg = rank & 7, cg = rank >> 3;
    const int i0 = 4 * rg, j0 = 4 * cg;  // halves at +0 and +32
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
#pragma unroll 1
    for (int l = 0; l < NMAX; l += 4) {
        float bq[8][4];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int j = j0 + (c & 3) + 32 * (c >> 2);
            const float4 v = *reinterpret_cast<const float4 *>(Bs + j * LD + l);
            bq[c][0] = v.x; bq[c][1] = v.y; bq[c][2] = v.z; bq[c][3] = v.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 a0 = *reinterpret_cast<const float4 *>(As + (l + u) * LD + i0);
            const float4 a1 = *reinterpret_cast<const float4 *>(As + (l + u) * LD + i0 + 32);
            const float af[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(af[r], bq[c][u], acc[r][c]);
        }
    }
    __syncthreads();
    float *Cs = As;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int j = j0 + (c & 3) + 32 * (c >> 2);
        *reinterpret_cast<float4 *>(Cs + j * LD + i0) = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
        *reinterpret_cast<float4 *>(Cs + j * LD + i0 + 32) = make_float4(acc[4][c], acc[5][c], acc[6][c], acc[7][c]);
    }
    __syncthreads();
    float *gc = C.p + (long long)b * C.s;
    for (int e = rank; e < n * q4; e += 64) {
        const int c = e / q4, q = e - c * q4;
        __stcs(reinterpret_cast<float4 *>(gc + c * n + 4 * q), *reinterpret_cast<const float4 *>(Cs + c * LD + 4 * q));
    }
}

template <typename K>
cudaError_t go(K kern, int grid, int threads, size_t smem, cudaStream_t st, int m, int n, int k, const Mat &A,
               const Mat &B, const Mat &C, int batch) {
    {
        cudaError_t e = prepare(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, threads, smem, st>>>(m, n, k, A, B, C, batch);
    return cudaPeekAtLastError();
}

constexpr size_t kMaxSmem = 227 * 1024;

int bucket(int d) { return d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : 64; }

// Team size of a scope for bucket N.
int team_of(int scope, int N) {
    if (scope == SCOPE_WARP) return 32;
    return N <= 16 ? 64 : (N <= 32 ? 128 : 256);
}

size_t smem_gemm(int m, int n, int k, Placement pl) {
    const int N = bucket(m > n ? (m > k ? m : k) : (n > k ? n : k));
    if (pl.scope == SCOPE_THREAD)
        return (size_t)32 * pl.pack * (odd_stride(m * k) + odd_stride(k * n) + odd_stride(m * n)) * 4;
    return (size_t)pl.pack * 2 * N * (N + 4) * 4;
}

}  // namespace

bool feasible_gemm(int m, int n, int k, Placement pl) {
    if (m < 1 || n < 1 || k < 1 || m > 64 || n > 64 || k > 64) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    const int N = bucket(m > n ? (m > k ? m : k) : (n > k ? n : k));
    if (pl.scope == SCOPE_THREAD && N > 8 && !(m == n && n == k && m <= 12)) return false;
    if (pl.scope != SCOPE_THREAD && team_of(pl.scope, N) * pl.pack > 256) return false;
    if (pl.scope == SCOPE_WARP && N < 8) return false;
    return smem_gemm(m, n, k, pl) <= kMaxSmem;
}

cudaError_t launch_gemm(int m, int n, int k, Mat A, Mat B, Mat C, int batch, Placement pl, cudaStream_t st) {
    if (!feasible_gemm(m, n, k, pl)) return cudaErrorInvalidConfiguration;
    const size_t smem = smem_gemm(m, n, k, pl);
    const int N = bucket(m > n ? (m > k ? m : k) : (n > k ? n : k));
    if (pl.scope == SCOPE_THREAD) {
        const int G = 32 * pl.pack;
        const int grid = ceil_div(batch, G);
        const size_t sm = A.layout == GLASS_LAYOUT_COLMAJOR ? smem : 0;
        if (m == n && n == k) {
            switch (n) {
                case 3: return go(k_gemm_thread<3, true>, grid, G, sm, st, m, n, k, A, B, C, batch);
                case 6: return go(k_gemm_thread<6, true>, grid, G, sm, st, m, n, k, A, B, C, batch);
                case 7: return go(k_gemm_thread<7, true>, grid, G, sm, st, m, n, k, A, B, C, batch);
                case 12: return go(k_gemm_thread<12, true>, grid, G, sm, st, m, n, k, A, B, C, batch);
                default: break;
            }
            if (n > 8) return go(k_gemm_thread<12, false>, grid, G, sm, st, m, n, k, A, B, C, batch);
        }
        if (N <= 4 && m <= 4 && n <= 4 && k <= 4)
            return go(k_gemm_thread<4, false>, grid, G, sm, st, m, n, k, A, B, C, batch);
        return go(k_gemm_thread<8, false>, grid, G, sm, st, m, n, k, A, B, C, batch);
    }
    const bool async_ok = pl.scope == SCOPE_BLOCK && pl.pack == 1 && m == n && n == k && (n & 3) == 0 && N >= 32 &&
                          A.packed() && B.packed() && C.packed() &&
                          ((reinterpret_cast<uintptr_t>(A.p) | reinterpret_cast<uintptr_t>(B.p) |
                            reinterpret_cast<uintptr_t>(C.p)) & 15) == 0;
    if (async_ok && m == 64) return launch_gemm_umma64(A.p, B.p, C.p, batch, st);
    // orders 16, 24 and 32, block x1 on packed aligned operands: the
    // streaming split-TF32 mma.sync kernel (each product within 3 * 2^-22 of
    // exact, FP32 accumulation: inside the FP32 bound 2k u |A||B| every FP32
    // GEMM here meets)
    if (pl.scope == SCOPE_BLOCK && pl.pack == 1 && m == n && n == k && (n == 16 || n == 24 || n == 32) &&
        A.packed() && B.packed() && C.packed() &&
        ((reinterpret_cast<uintptr_t>(A.p) | reinterpret_cast<uintptr_t>(B.p) | reinterpret_cast<uintptr_t>(C.p)) &
         15) == 0)
        return launch_gemm_tc(n, GLASS_MATH_3XTF32_TC, A.p, B.p, C.p, batch, st);
    if (async_ok) {
        const size_t sm = (size_t)2 * N * (N + 4) * 4;
        cudaError_t e;
        if (N == 32) {
            if ((e = prepare(k_gemm_async<32, 64>, sm)) != cudaSuccess) return e;
            k_gemm_async<32, 64><<<batch, 64, sm, st>>>(n, A, B, C, batch);
        } else {
            if ((e = prepare(k_gemm_async8<64>, sm)) != cudaSuccess) return e;
            k_gemm_async8<64><<<batch, 64, sm, st>>>(n, A, B, C, batch);
        }
        return cudaPeekAtLastError();
    }
    const int T = team_of(pl.scope, N);
    const int grid = ceil_div(batch, pl.pack);
    const int th = T * pl.pack;
#define GL_G(NN, TT) go(k_gemm_team<NN, TT>, grid, th, smem, st, m, n, k, A, B, C, batch)
    if (N == 8) return T == 32 ? GL_G(8, 32) : GL_G(8, 64);
    if (N == 16) return T == 32 ? GL_G(16, 32) : GL_G(16, 64);
    if (N == 32) return T == 32 ? GL_G(32, 32) : GL_G(32, 128);
    return T == 32 ? GL_G(64, 32) : GL_G(64, 256);
#undef GL_G
}

}  // namespace glass
