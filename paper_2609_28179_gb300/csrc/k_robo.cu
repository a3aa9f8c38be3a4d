// k_robo.cu -- robotics operations of the paper's placement table (Sec.
// IV-E, Table II): quaternion and SE(3) retractions, quaternion error,
// spatial-motion cross product, symmetric 3x3 eigen-decomposition, 3x3 SVD,
// closest rotation, argmax and softmax, at thread, warp and block scope.
//
// Conventions (fixed by the interface, as the paper requires of every
// operation; include/glass.h states them): quaternions (w, x, y, z),
// Hamilton product; rotation vectors; twists and motion vectors with the
// linear part first; right perturbations; 4x4 and 3x3 matrices column-major.
//
// Thread scope computes one problem per thread (32*pack per CTA).  argmax
// and softmax also run at warp and block scope, the n elements of a problem
// spread over a warp or a 64-thread team and reduced with shuffles (and
// shared memory across warps).  The element-wise operations are thread scope
// only: one problem is a short serial chain of dependent arithmetic with
// nothing for a team to share, so a team placement would leave all but one
// lane idle.
#include <math.h>

#include "common.cuh"

namespace glass {
namespace {

// ------------------------------------------------------------ math helpers
__device__ __forceinline__ void qmul(const float *a, const float *b, float *o) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Exp of a rotation vector: (cos t/2, sin(t/2) d / t); sin(t/2)/t -> 1/2.
__device__ __forceinline__ void qexp(const float *d, float *q) {
    const float t = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    float s, c;
    sincosf(0.5f * t, &s, &c);
    const float f = t > 0.f ? s / t : 0.5f;
    q[0] = c;
    q[1] = f * d[0];
    q[2] = f * d[1];
    q[3] = f * d[2];
}

// Log of a unit quaternion on the w >= 0 hemisphere: 2 atan2(|v|, w) v / |v|.
__device__ __forceinline__ void qlog(const float *qin, float *d) {
    const float sg = qin[0] < 0.f ? -1.f : 1.f;
    const float w = sg * qin[0], x = sg * qin[1], y = sg * qin[2], z = sg * qin[3];
    const float nv = sqrtf(x * x + y * y + z * z);
    const float f = nv > 0.f ? 2.f * atan2f(nv, w) / nv : 2.f / w;
    d[0] = f * x;
    d[1] = f * y;
    d[2] = f * z;
}

__device__ __forceinline__ void cross3(const float *a, const float *b, float *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Exp of a twist (rho, phi): R = I + a S + b S^2, V = I + b S + c S^2 with
// S = [phi]x, a = sin t / t, b = 2 sin^2(t/2) / t^2, c = (t - sin t) / t^3
// (its Taylor series below t = 0.5, where the difference cancels in FP32).
__device__ __forceinline__ void se3_exp(const float *xi, float *R, float *tv) {
    const float *rho = xi, *phi = xi + 3;
    const float t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2], t = sqrtf(t2);
    float a = 1.f, b = 0.5f, c;
    if (t > 0.f) {
        float s, co, sh, ch;
        sincosf(t, &s, &co);
        sincosf(0.5f * t, &sh, &ch);
        a = s / t;
        b = 2.f * sh * sh / t2;
    }
    if (t < 0.5f)
        c = 1.f / 6.f + t2 * (-1.f / 120.f + t2 * (1.f / 5040.f + t2 * (-1.f / 362880.f + t2 * (1.f / 39916800.f))));
    else
        c = (t - sinf(t)) / (t2 * t);
    const float S[9] = {0.f, phi[2], -phi[1], -phi[2], 0.f, phi[0], phi[1], -phi[0], 0.f};
    float S2[9];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i)
            S2[j * 3 + i] = S[i] * S[j * 3] + S[3 + i] * S[j * 3 + 1] + S[6 + i] * S[j * 3 + 2];
    float V[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float id = (k % 4 == 0) ? 1.f : 0.f;
        R[k] = id + a * S[k] + b * S2[k];
        V[k] = id + b * S[k] + c * S2[k];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) tv[i] = V[i] * rho[0] + V[3 + i] * rho[1] + V[6 + i] * rho[2];
}

// Cyclic Jacobi on a symmetric 3x3 (column-major), FP32, until the
// off-diagonal mass is negligible (at most 12 sweeps); eigenvalues
// ascending, eigenvector columns with their largest component positive.
__device__ __forceinline__ void eig3(const float *Ain, float *w, float *Vout) {
    float A[9], V[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
#pragma unroll
    for (int k = 0; k < 9; ++k) A[k] = Ain[k];
    const float scale = A[0] * A[0] + A[4] * A[4] + A[8] * A[8] + 2.f * (A[3] * A[3] + A[6] * A[6] + A[7] * A[7]);
    for (int sweep = 0; sweep < 12; ++sweep) {
        const float off = A[3] * A[3] + A[6] * A[6] + A[7] * A[7];
        if (!(off > 1e-16f * scale)) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const float apq = A[q * 3 + p];
            if (apq == 0.f) continue;
            const float app = A[p * 3 + p], aqq = A[q * 3 + q];
            const float theta = (aqq - app) / (2.f * apq);
            const float tt = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = 1.f / sqrtf(tt * tt + 1.f), s = tt * c;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float akp = A[p * 3 + k], akq = A[q * 3 + k];
                A[p * 3 + k] = c * akp - s * akq;
                A[q * 3 + k] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float apk = A[k * 3 + p], aqk = A[k * 3 + q];
                A[k * 3 + p] = c * apk - s * aqk;
                A[k * 3 + q] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[p * 3 + k], vkq = V[q * 3 + k];
                V[p * 3 + k] = c * vkp - s * vkq;
                V[q * 3 + k] = s * vkp + c * vkq;
            }
        }
    }
    // sort ascending: three compare-exchanges of (eigenvalue, column) pairs
    float d[3] = {A[0], A[4], A[8]};
#define CX(i, j)                                                                       \
    if (d[j] < d[i]) {                                                                 \
        const float td = d[i]; d[i] = d[j]; d[j] = td;                                 \
        _Pragma("unroll") for (int k = 0; k < 3; ++k) {                                \
            const float tv = V[i * 3 + k]; V[i * 3 + k] = V[j * 3 + k]; V[j * 3 + k] = tv; \
        }                                                                              \
    }
    CX(0, 1) CX(1, 2) CX(0, 1)
#undef CX
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        w[c] = d[c];
        const float v0 = V[c * 3], v1 = V[c * 3 + 1], v2 = V[c * 3 + 2];
        const float big = fabsf(v1) > fabsf(v0) ? (fabsf(v2) > fabsf(v1) ? v2 : v1) : (fabsf(v2) > fabsf(v0) ? v2 : v0);
        const float sg = big < 0.f ? -1.f : 1.f;
        Vout[c * 3] = sg * v0;
        Vout[c * 3 + 1] = sg * v1;
        Vout[c * 3 + 2] = sg * v2;
    }
}

// One-sided Jacobi SVD of a 3x3 (column-major): rotate column pairs of
// W = M V until orthogonal; s_i = |w_i| descending, U = W / s; a zero s3
// gets u3 = u1 x u2 (and a zero s2 an arbitrary unit vector orthogonal to u1).
__device__ __forceinline__ void svd3(const float *M, float *U, float *s, float *V) {
    float W[9], Vm[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = M[k];
    for (int sweep = 0; sweep < 12; ++sweep) {
        bool rotated = false;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                al = fmaf(W[p * 3 + k], W[p * 3 + k], al);
                be = fmaf(W[q * 3 + k], W[q * 3 + k], be);
                ga = fmaf(W[p * 3 + k], W[q * 3 + k], ga);
            }
            if (!(fabsf(ga) > 1e-7f * sqrtf(al * be))) continue;
            rotated = true;
            const float zeta = (be - al) / (2.f * ga);
            const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
            const float c = 1.f / sqrtf(1.f + tt * tt), sn = c * tt;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float wp = W[p * 3 + k], wq = W[q * 3 + k];
                W[p * 3 + k] = c * wp - sn * wq;
                W[q * 3 + k] = sn * wp + c * wq;
                const float vp = Vm[p * 3 + k], vq = Vm[q * 3 + k];
                Vm[p * 3 + k] = c * vp - sn * vq;
                Vm[q * 3 + k] = sn * vp + c * vq;
            }
        }
        if (!rotated) break;
    }
    float n[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) n[c] = sqrtf(W[c * 3] * W[c * 3] + W[c * 3 + 1] * W[c * 3 + 1] + W[c * 3 + 2] * W[c * 3 + 2]);
    // sort descending: compare-exchanges of (norm, column of W, column of V)
#define CX(i, j)                                                                          \
    if (n[j] > n[i]) {                                                                    \
        const float tn = n[i]; n[i] = n[j]; n[j] = tn;                                    \
        _Pragma("unroll") for (int k = 0; k < 3; ++k) {                                   \
            const float tw = W[i * 3 + k]; W[i * 3 + k] = W[j * 3 + k]; W[j * 3 + k] = tw;   \
            const float tv = Vm[i * 3 + k]; Vm[i * 3 + k] = Vm[j * 3 + k]; Vm[j * 3 + k] = tv; \
        }                                                                                 \
    }
    CX(0, 1) CX(1, 2) CX(0, 1)
#undef CX
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s[c] = n[c];
        const float inv = s[c] > 0.f ? 1.f / s[c] : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            U[c * 3 + k] = W[c * 3 + k] * inv;
            V[c * 3 + k] = Vm[c * 3 + k];
        }
    }
    if (!(s[1] > 1e-7f * s[0])) {  // rank one (or zero): any unit vector orthogonal to u1
        const float e[3] = {fabsf(U[0]) < 0.5f ? 1.f : 0.f, fabsf(U[0]) < 0.5f ? 0.f : 1.f, 0.f};
        float t[3];
        cross3(U, e, t);
        const float tn = rsqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
        U[3] = t[0] * tn;
        U[4] = t[1] * tn;
        U[5] = t[2] * tn;
        if (!(s[0] > 0.f)) {  // zero matrix: U = I
            U[0] = 1.f, U[1] = 0.f, U[2] = 0.f, U[3] = 0.f, U[4] = 1.f, U[5] = 0.f;
        }
    }
    if (!(s[2] > 1e-7f * s[0])) cross3(U, U + 3, U + 6);
}

__device__ __forceinline__ float det3(const float *A) {
    return A[0] * (A[4] * A[8] - A[7] * A[5]) - A[3] * (A[1] * A[8] - A[7] * A[2]) + A[6] * (A[1] * A[5] - A[4] * A[2]);
}

// --------------------------------------------------------------- operations
struct QuatRetract {
    const float *q, *d;
    float *out;
    __device__ void operator()(long long b) const {
        const float4 qq = reinterpret_cast<const float4 *>(q)[b];
        const float a[4] = {qq.x, qq.y, qq.z, qq.w};
        const float dd[3] = {d[3 * b], d[3 * b + 1], d[3 * b + 2]};
        float e[4], o[4];
        qexp(dd, e);
        qmul(a, e, o);
        reinterpret_cast<float4 *>(out)[b] = make_float4(o[0], o[1], o[2], o[3]);
    }
};

struct QuatError {
    const float *q1, *q2;
    float *out;
    __device__ void operator()(long long b) const {
        const float4 a = reinterpret_cast<const float4 *>(q1)[b];
        const float4 c = reinterpret_cast<const float4 *>(q2)[b];
        const float ca[4] = {a.x, -a.y, -a.z, -a.w}, cb[4] = {c.x, c.y, c.z, c.w};
        float r[4], e[3];
        qmul(ca, cb, r);
        qlog(r, e);
        out[3 * b] = e[0];
        out[3 * b + 1] = e[1];
        out[3 * b + 2] = e[2];
    }
};

struct Se3Retract {
    const float *T, *xi;
    float *out;
    __device__ void operator()(long long b) const {
        const float4 *t4 = reinterpret_cast<const float4 *>(T) + 4 * b;
        float t[16];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 v = t4[c];
            t[4 * c] = v.x, t[4 * c + 1] = v.y, t[4 * c + 2] = v.z, t[4 * c + 3] = v.w;
        }
        float x[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) x[i] = xi[6 * b + i];
        float R[9], tv[3];
        se3_exp(x, R, tv);
        // [Rt tt; 0 1] [R tv; 0 1] = [Rt R, Rt tv + tt; 0 1]
        float4 *o4 = reinterpret_cast<float4 *>(out) + 4 * b;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float o[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) o[i] = t[i] * R[j * 3] + t[4 + i] * R[j * 3 + 1] + t[8 + i] * R[j * 3 + 2];
            o4[j] = make_float4(o[0], o[1], o[2], 0.f);
        }
        float o[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) o[i] = t[i] * tv[0] + t[4 + i] * tv[1] + t[8 + i] * tv[2] + t[12 + i];
        o4[3] = make_float4(o[0], o[1], o[2], 1.f);
    }
};

struct MotionCross {
    const float *v, *m;
    float *out;
    __device__ void operator()(long long b) const {
        float a[6], c[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) a[i] = v[6 * b + i], c[i] = m[6 * b + i];
        float c1[3], c2[3], c3[3];
        cross3(a + 3, c, c1);
        cross3(a, c + 3, c2);
        cross3(a + 3, c + 3, c3);
#pragma unroll
        for (int i = 0; i < 3; ++i) out[6 * b + i] = c1[i] + c2[i], out[6 * b + 3 + i] = c3[i];
    }
};

struct Eig3 {
    const float *A;
    float *w, *V;
    __device__ void operator()(long long b) const {
        float a[9], ww[3], vv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) a[i] = A[9 * b + i];
        eig3(a, ww, vv);
#pragma unroll
        for (int i = 0; i < 3; ++i) w[3 * b + i] = ww[i];
#pragma unroll
        for (int i = 0; i < 9; ++i) V[9 * b + i] = vv[i];
    }
};

struct Svd3 {
    const float *M;
    float *U, *S, *V;
    __device__ void operator()(long long b) const {
        float a[9], u[9], s[3], v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) a[i] = M[9 * b + i];
        svd3(a, u, s, v);
#pragma unroll
        for (int i = 0; i < 9; ++i) U[9 * b + i] = u[i], V[9 * b + i] = v[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) S[3 * b + i] = s[i];
    }
};

struct ClosestRotation {
    const float *M;
    float *R;
    __device__ void operator()(long long b) const {
        float a[9], u[9], s[3], v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) a[i] = M[9 * b + i];
        svd3(a, u, s, v);
        const float d = det3(u) * det3(v) < 0.f ? -1.f : 1.f;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                R[9 * b + j * 3 + i] = u[i] * v[j] + u[3 + i] * v[3 + j] + d * u[6 + i] * v[6 + j];
    }
};

template <class Op>
__global__ void __launch_bounds__(256) k_elementwise(Op op, int batch) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    op(b);
}

// ------------------------------------------------------------ reductions
struct Best {
    float v;
    int i;
};
__device__ __forceinline__ Best better(Best a, Best b) {
    return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

template <int T>
__global__ void __launch_bounds__(256) k_argmax(int n, const float *x, long long sx, int *idx, int batch) {
    __shared__ Best part[8];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const long long b = (long long)blockIdx.x * (blockDim.x / T) + team;
    if (b >= batch) return;  // whole team
    const float *v = x + b * sx;
    Best best{-INFINITY, 0x7fffffff};
    for (int i = rank; i < n; i += T) best = better(best, Best{v[i], i});
    if constexpr (T > 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const Best other{__shfl_xor_sync(GLASS_FULL_MASK, best.v, o), __shfl_xor_sync(GLASS_FULL_MASK, best.i, o)};
            best = better(best, other);
        }
    }
    if constexpr (T > 32) {
        const int w = threadIdx.x >> 5;
        if ((rank & 31) == 0) part[w] = best;
        team_sync<T>(1 + team);
        if (rank == 0)
            for (int k = 1; k < T / 32; ++k) best = better(best, part[w + k]);
    }
    if (rank == 0) idx[b] = best.i == 0x7fffffff ? 0 : best.i;
}

template <int T>
__global__ void __launch_bounds__(256) k_softmax(int n, const float *x, long long sx, float *y, long long sy,
                                                 int batch) {
    __shared__ float part[2][8];
    const int team = threadIdx.x / T, rank = threadIdx.x % T;
    const long long b = (long long)blockIdx.x * (blockDim.x / T) + team;
    if (b >= batch) return;  // whole team
    const float *v = x + b * sx;
    float *o = y + b * sy;
    float mx = -INFINITY;
    for (int i = rank; i < n; i += T) mx = fmaxf(mx, v[i]);
    if (T > 1) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(GLASS_FULL_MASK, mx, s));
        if (T > 32) {
            const int w = threadIdx.x >> 5, w0 = (threadIdx.x - rank) >> 5;
            if ((rank & 31) == 0) part[0][w] = mx;
            team_sync<T>(1 + team);
            for (int k = 0; k < T / 32; ++k) mx = fmaxf(mx, part[0][w0 + k]);
        }
    }
    float sum = 0.f;
    for (int i = rank; i < n; i += T) sum += expf(v[i] - mx);
    if (T > 1) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) sum += __shfl_xor_sync(GLASS_FULL_MASK, sum, s);
        if (T > 32) {
            const int w = threadIdx.x >> 5, w0 = (threadIdx.x - rank) >> 5;
            if ((rank & 31) == 0) part[1][w] = sum;
            team_sync<T>(1 + team);
            sum = 0.f;
            for (int k = 0; k < T / 32; ++k) sum += part[1][w0 + k];
        }
    }
    const float inv = 1.f / sum;
    for (int i = rank; i < n; i += T) o[i] = expf(v[i] - mx) * inv;
}

template <class Op>
cudaError_t launch_elementwise(Op op, int batch, Placement pl, cudaStream_t st) {
    const int th = 32 * pl.pack;  // thread scope: one problem per thread
    k_elementwise<Op><<<ceil_div(batch, th), th, 0, st>>>(op, batch);
    return cudaPeekAtLastError();
}

}  // namespace

bool feasible_robo(int op, int n, Placement pl) {
    if (pl.pack != 1 && pl.pack != 2 && pl.pack != 4 && pl.pack != 8) return false;
    if (pl.scope == SCOPE_BLOCK && pl.pack > 4) return false;
    if (pl.scope < SCOPE_THREAD || pl.scope > SCOPE_BLOCK) return false;
    if (op == ROBO_ARGMAX || op == ROBO_SOFTMAX) return n >= 1;
    return pl.scope == SCOPE_THREAD;  // element-wise: nothing for a team to share
}

cudaError_t launch_robo(int op, int n, const float *a, const float *b, long long sa, float *o1, float *o2, float *o3,
                        long long so, int *idx, int batch, Placement pl, cudaStream_t st) {
    if (!feasible_robo(op, n, pl)) return cudaErrorInvalidConfiguration;
    switch (op) {
        case ROBO_QUAT_RETRACT: return launch_elementwise(QuatRetract{a, b, o1}, batch, pl, st);
        case ROBO_QUAT_ERROR: return launch_elementwise(QuatError{a, b, o1}, batch, pl, st);
        case ROBO_SE3_RETRACT: return launch_elementwise(Se3Retract{a, b, o1}, batch, pl, st);
        case ROBO_MOTION_CROSS: return launch_elementwise(MotionCross{a, b, o1}, batch, pl, st);
        case ROBO_EIG3: return launch_elementwise(Eig3{a, o1, o2}, batch, pl, st);
        case ROBO_SVD3: return launch_elementwise(Svd3{a, o1, o2, o3}, batch, pl, st);
        case ROBO_CLOSEST_ROTATION: return launch_elementwise(ClosestRotation{a, o1}, batch, pl, st);
        default: break;
    }
    const int th = pl.scope == SCOPE_THREAD ? 32 * pl.pack : (pl.scope == SCOPE_WARP ? 32 : 64) * pl.pack;
    const int per = pl.scope == SCOPE_THREAD ? th : pl.pack;
    const int grid = ceil_div(batch, per);
    if (op == ROBO_ARGMAX) {
        if (pl.scope == SCOPE_THREAD) k_argmax<1><<<grid, th, 0, st>>>(n, a, sa, idx, batch);
        else if (pl.scope == SCOPE_WARP) k_argmax<32><<<grid, th, 0, st>>>(n, a, sa, idx, batch);
        else k_argmax<64><<<grid, th, 0, st>>>(n, a, sa, idx, batch);
    } else {
        if (pl.scope == SCOPE_THREAD) k_softmax<1><<<grid, th, 0, st>>>(n, a, sa, o1, so, batch);
        else if (pl.scope == SCOPE_WARP) k_softmax<32><<<grid, th, 0, st>>>(n, a, sa, o1, so, batch);
        else k_softmax<64><<<grid, th, 0, st>>>(n, a, sa, o1, so, batch);
    }
    return cudaPeekAtLastError();
}

}  // namespace glass
