// k_geom.cu -- batched rotation-chain composition and SE(3) apply
// (Sec. III-B: SO(3) / SE(3) maps), plus the 32-problem interleaved layout
// converters.
//
// A chain T_0 ... T_{c-1} is composed left to right.  Thread scope composes
// serially; warp and block scope compose with a binary tree of 3x3 (or 3x4
// affine) products across lanes -- the product is associative, so only the
// rounding order differs from the serial definition.  SE(3) apply then
// streams the points with 16-byte loads (4 points = 3 float4).
#include "common.cuh"

namespace glass {
namespace {

// 3x4 affine [R | t] in column-major 12 floats: R at 0..8, t at 9..11.
struct Aff {
    float m[12];
};

__device__ __forceinline__ void aff_identity(Aff &a) {
#pragma unroll
    for (int u = 0; u < 12; ++u) a.m[u] = 0.f;
    a.m[0] = a.m[4] = a.m[8] = 1.f;
}

// x <- x * y  (rotation part only when ROT_ONLY)
template <bool ROT_ONLY>
__device__ __forceinline__ void aff_mul(Aff &x, const Aff &y) {
    Aff z;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            z.m[j * 3 + i] = fmaf(x.m[i], y.m[j * 3], fmaf(x.m[3 + i], y.m[j * 3 + 1], x.m[6 + i] * y.m[j * 3 + 2]));
    if (!ROT_ONLY) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
            z.m[9 + i] = fmaf(x.m[i], y.m[9], fmaf(x.m[3 + i], y.m[10], fmaf(x.m[6 + i], y.m[11], x.m[9 + i])));
    } else {
        z.m[9] = z.m[10] = z.m[11] = 0.f;
    }
    x = z;
}

// Element u (0..11) of chain entry c: a 3x3 rotation (9 floats) or the top
// three rows of a 4x4 transform (16 floats, column-major).
template <bool ROT>
__device__ __forceinline__ float chain_elem(const float *p, int c, int u) {
    if (ROT) return u < 9 ? p[c * 9 + u] : 0.f;
    const int col = u < 9 ? u / 3 : 3, row = u < 9 ? u - 3 * (u / 3) : u - 9;
    return p[c * 16 + col * 4 + row];
}

template <bool ROT>
__device__ __forceinline__ void load_aff(Aff &a, const float *p, int c) {
    if (!ROT && (reinterpret_cast<uintptr_t>(p + c * 16) & 15) == 0) {
        // a 4 x 4 transform is four 16-byte columns; the bottom row is not used
        const float4 *q = reinterpret_cast<const float4 *>(p + c * 16);
#pragma unroll
        for (int col = 0; col < 4; ++col) {
            const float4 v = __ldg(q + col);
            a.m[3 * col] = v.x;
            a.m[3 * col + 1] = v.y;
            a.m[3 * col + 2] = v.z;
        }
        return;
    }
#pragma unroll
    for (int u = 0; u < 12; ++u) a.m[u] = chain_elem<ROT>(p, c, u);
}

__device__ __forceinline__ Aff shfl_down_aff(const Aff &a, int d) {
    Aff r;
#pragma unroll
    for (int u = 0; u < 12; ++u) r.m[u] = __shfl_down_sync(GLASS_FULL_MASK, a.m[u], d);
    return r;
}

// Warp tree over entries lane, lane+32 (chain <= 64): result in lane 0.
template <bool ROT>
__device__ __forceinline__ Aff warp_compose(const float *p, int chain) {
    const int lane = threadIdx.x & 31;
    Aff acc;
    const int c0 = 2 * lane;
    if (c0 < chain) load_aff<ROT>(acc, p, c0);
    else aff_identity(acc);
    if (c0 + 1 < chain) {
        Aff y;
        load_aff<ROT>(y, p, c0 + 1);
        aff_mul<ROT>(acc, y);
    }
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const Aff y = shfl_down_aff(acc, s);
        if ((lane & (2 * s - 1)) == 0) aff_mul<ROT>(acc, y);
    }
    return acc;
}

__device__ __forceinline__ void apply_point(const Aff &T, float x, float y, float z, float &qx, float &qy,
                                            float &qz) {
    qx = fmaf(T.m[0], x, fmaf(T.m[3], y, fmaf(T.m[6], z, T.m[9])));
    qy = fmaf(T.m[1], x, fmaf(T.m[4], y, fmaf(T.m[7], z, T.m[10])));
    qz = fmaf(T.m[2], x, fmaf(T.m[5], y, fmaf(T.m[8], z, T.m[11])));
}

// Four points as 3 float4 (x0 y0 z0 x1 | y1 z1 x2 y2 | z2 x3 y3 z3).
struct Quad {
    float4 a, b, c;
};

__device__ __forceinline__ Quad load_quad(const float *P, int g) {
    const float4 *src = reinterpret_cast<const float4 *>(P) + 3 * g;
    return Quad{__ldcs(src), __ldcs(src + 1), __ldcs(src + 2)};
}

__device__ __forceinline__ void apply_quad(const Aff &T, const Quad &v, float *Q, int g) {
    float4 o0, o1, o2;
    apply_point(T, v.a.x, v.a.y, v.a.z, o0.x, o0.y, o0.z);
    apply_point(T, v.a.w, v.b.x, v.b.y, o0.w, o1.x, o1.y);
    apply_point(T, v.b.z, v.b.w, v.c.x, o1.z, o1.w, o2.x);
    apply_point(T, v.c.y, v.c.z, v.c.w, o2.y, o2.z, o2.w);
    float4 *dst = reinterpret_cast<float4 *>(Q) + 3 * g;
    __stcs(dst, o0);
    __stcs(dst + 1, o1);
    __stcs(dst + 2, o2);
}

__device__ __forceinline__ bool quads_ok(const float *P, const float *Q) {
    return ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(Q)) & 15) == 0;
}

// Stream npts points of one problem with `nthr` cooperating threads, from
// group g0 (of four points) on: four groups per step, all their loads
// issued before any is transformed; a ragged tail point by point.
__device__ __forceinline__ void stream_points(const Aff &T, const float *P, float *Q, int npts, int rank, int nthr,
                                              int g0 = -1) {
    const int ng = quads_ok(P, Q) ? npts / 4 : 0;
    int g = g0 < 0 ? rank : g0;
    for (; g + 3 * nthr < ng; g += 4 * nthr) {
        Quad v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = load_quad(P, g + k * nthr);
#pragma unroll
        for (int k = 0; k < 4; ++k) apply_quad(T, v[k], Q, g + k * nthr);
    }
    for (; g < ng; g += nthr) apply_quad(T, load_quad(P, g), Q, g);
    for (int i = 4 * ng + rank; i < npts; i += nthr) {
        float qx, qy, qz;
        apply_point(T, P[3 * i], P[3 * i + 1], P[3 * i + 2], qx, qy, qz);
        Q[3 * i] = qx;
        Q[3 * i + 1] = qy;
        Q[3 * i + 2] = qz;
    }
}

// ---------------------------------------------------------------- kernels
// OP: 0 = rot3 compose (out: 9 floats), 1 = se3 apply
template <int OP>
__global__ void __launch_bounds__(256) k_geom_thread(int chain, Mat T, int npts, Mat P, Mat Q, int batch) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    constexpr bool ROT = OP == 0;
    const float *p = T.p + (long long)b * T.s;
    Aff acc;
    load_aff<ROT>(acc, p, 0);
    for (int c = 1; c < chain; ++c) {
        Aff y;
        load_aff<ROT>(y, p, c);
        aff_mul<ROT>(acc, y);
    }
    if (OP == 0) {
        float *r = Q.p + (long long)b * Q.s;
#pragma unroll
        for (int u = 0; u < 9; ++u) r[u] = acc.m[u];
    } else {
        stream_points(acc, P.p + (long long)b * P.s, Q.p + (long long)b * Q.s, npts, 0, 1);
    }
}

template <int OP>
__global__ void __launch_bounds__(256) k_geom_warp(int chain, Mat T, int npts, Mat P, Mat Q, int batch) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= batch) return;
    constexpr bool ROT = OP == 0;
    // SE(3): this lane's first two groups of points are already on their way
    // while the warp composes the chain
    const float *pb = OP == 1 ? P.p + (long long)b * P.s : nullptr;
    float *qb = OP == 1 ? Q.p + (long long)b * Q.s : nullptr;
    const bool pre = OP == 1 && quads_ok(pb, qb) && lane + 32 < npts / 4;
    Quad first{}, second{};
    if (pre) {
        first = load_quad(pb, lane);
        second = load_quad(pb, lane + 32);
    }
    Aff acc = warp_compose<ROT>(T.p + (long long)b * T.s, chain);
#pragma unroll
    for (int u = 0; u < 12; ++u) acc.m[u] = __shfl_sync(GLASS_FULL_MASK, acc.m[u], 0);
    if (OP == 0) {
        float *r = Q.p + (long long)b * Q.s;
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 9; ++u) r[u] = acc.m[u];
        }
    } else {
        if (pre) {
            apply_quad(acc, first, qb, lane);
            apply_quad(acc, second, qb, lane + 32);
        }
        stream_points(acc, pb, qb, npts, lane, 32, pre ? lane + 64 : lane);
    }
}

// Block scope: team of TB threads; the first warp composes, all stream.
template <int OP, int TB>
__global__ void __launch_bounds__(1024) k_geom_block(int chain, Mat T, int npts, Mat P, Mat Q, int batch) {
    __shared__ float sh[8][12];
    const int team = threadIdx.x / TB, rank = threadIdx.x % TB;
    const int P_ = blockDim.x / TB;
    const int b = blockIdx.x * P_ + team;
    const int bar = 1 + team;
    if (b >= batch) return;
    constexpr bool ROT = OP == 0;
    if (rank < 32) {
        const Aff acc = warp_compose<ROT>(T.p + (long long)b * T.s, chain);
        if (rank == 0)
#pragma unroll
            for (int u = 0; u < 12; ++u) sh[team][u] = acc.m[u];
    }
    team_sync<TB>(bar);
    Aff acc;
#pragma unroll
    for (int u = 0; u < 12; ++u) acc.m[u] = sh[team][u];
    if (OP == 0) {
        if (rank < 9) Q.p[(long long)b * Q.s + rank] = sh[team][rank];
    } else {
        stream_points(acc, P.p + (long long)b * P.s, Q.p + (long long)b * Q.s, npts, rank, TB);
    }
}

// 32 x 32 tile transpose between packed column-major and interleaved-32.
template <bool TO>
__global__ void __launch_bounds__(1024) k_interleave(int per, const float *src, float *dst, int batch) {
    __shared__ float tile[32][33];
    const int e0 = blockIdx.x * 32, g = blockIdx.y;  // 32-problem group g
    const int tx = threadIdx.x, ty = threadIdx.y;    // 32 x 32 threads
    // TO: src[b*per + e] -> dst[(g*per + e)*32 + b%32]
    if (TO) {
        const int b = g * 32 + ty, e = e0 + tx;
        tile[ty][tx] = (b < batch && e < per) ? src[(long long)b * per + e] : 0.f;
        __syncthreads();
        const int e2 = e0 + ty;
        if (e2 < per) dst[((long long)g * per + e2) * 32 + tx] = tile[tx][ty];
    } else {
        const int e = e0 + ty;
        tile[ty][tx] = (e < per) ? src[((long long)g * per + e) * 32 + tx] : 0.f;
        __syncthreads();
        const int b = g * 32 + ty, e2 = e0 + tx;
        if (b < batch && e2 < per) dst[(long long)b * per + e2] = tile[tx][ty];
    }
}

template <typename K>
cudaError_t go(K kern, int grid, int threads, cudaStream_t st, int chain, const Mat &T, int npts, const Mat &P,
               const Mat &Q, int batch) {
    kern<<<grid, threads, 0, st>>>(chain, T, npts, P, Q, batch);
    return cudaPeekAtLastError();
}

int geom_team(int op) { return op == 0 ? 64 : 256; }

}  // namespace

bool feasible_geom(int op, int chain, Placement pl) {
    if (chain < 1 || chain > 64) return false;
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (pl.scope == SCOPE_BLOCK && geom_team(op) * pl.pack > 1024) return false;
    return pl.scope >= SCOPE_THREAD && pl.scope <= SCOPE_BLOCK;
}

cudaError_t launch_rot3(int chain, Mat Rs, Mat R, int batch, Placement pl, cudaStream_t st) {
    if (!feasible_geom(0, chain, pl)) return cudaErrorInvalidConfiguration;
    Mat none = R;
    if (pl.scope == SCOPE_THREAD) return go(k_geom_thread<0>, ceil_div(batch, 32 * pl.pack), 32 * pl.pack, st, chain, Rs, 0, none, R, batch);
    if (pl.scope == SCOPE_WARP) return go(k_geom_warp<0>, ceil_div(batch, pl.pack), 32 * pl.pack, st, chain, Rs, 0, none, R, batch);
    return go(k_geom_block<0, 64>, ceil_div(batch, pl.pack), 64 * pl.pack, st, chain, Rs, 0, none, R, batch);
}

cudaError_t launch_se3(int chain, Mat T, int npts, Mat P, Mat Q, int batch, Placement pl, cudaStream_t st) {
    if (!feasible_geom(1, chain, pl)) return cudaErrorInvalidConfiguration;
    if (pl.scope == SCOPE_THREAD) return go(k_geom_thread<1>, ceil_div(batch, 32 * pl.pack), 32 * pl.pack, st, chain, T, npts, P, Q, batch);
    if (pl.scope == SCOPE_WARP) return go(k_geom_warp<1>, ceil_div(batch, pl.pack), 32 * pl.pack, st, chain, T, npts, P, Q, batch);
    return go(k_geom_block<1, 256>, ceil_div(batch, pl.pack), 256 * pl.pack, st, chain, T, npts, P, Q, batch);
}

cudaError_t launch_to_interleaved(int rows, int cols, const float *src, float *dst, int batch, cudaStream_t st) {
    const int per = rows * cols;
    dim3 grid(ceil_div(per, 32), ceil_div(batch, 32)), block(32, 32);
    k_interleave<true><<<grid, block, 0, st>>>(per, src, dst, batch);
    return cudaPeekAtLastError();
}

cudaError_t launch_from_interleaved(int rows, int cols, const float *src, float *dst, int batch, cudaStream_t st) {
    const int per = rows * cols;
    dim3 grid(ceil_div(per, 32), ceil_div(batch, 32)), block(32, 32);
    k_interleave<false><<<grid, block, 0, st>>>(per, src, dst, batch);
    return cudaPeekAtLastError();
}

}  // namespace glass
