// k_mlp.cu -- training and inference kernels of the learned placement cost
// model: a perceptron din -> 64 -> 64 -> 12 with ReLU, fitted to the log
// latency of the 12 placements by masked mean-squared error and Adam.  (The
// paper selects placements by exhaustive offline measurement only,
// Sec. III-A; the model predicts placements for shapes off the measured
// grid.)
//
// Weights (row-major, out x in), packed: W1[64][din] b1[64] W2[64][64] b2[64]
// W3[12][64] b3[12].
//
// Forward: one row per thread, weights broadcast from shared memory.
// Loss/gradient: a CTA takes a tile of 64 rows, keeps each row's
// activations and deltas in shared memory, and forms the weight-gradient
// contributions of its tile as dot products over the tile's rows; the
// per-CTA partial gradients go to the caller's workspace and a second kernel
// sums them in a fixed order (deterministic), dividing by max(1, sum mask).
#include "common.cuh"

namespace glass {
namespace {

constexpr int H = 64;
constexpr int DOUT = 12;
constexpr int DIN = 8;
constexpr int NP = H * DIN + H + H * H + H + DOUT * H + DOUT;  // 5516
constexpr int OW1 = 0, OB1 = OW1 + H * DIN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + DOUT * H;
constexpr int TILE = 64;  // rows per CTA in the gradient kernel

__device__ __forceinline__ void forward_row(const float *w, const float *x, float *h1, float *h2, float *y) {
#pragma unroll 4
    for (int o = 0; o < H; ++o) {
        float s = w[OB1 + o];
#pragma unroll
        for (int i = 0; i < DIN; ++i) s = fmaf(w[OW1 + o * DIN + i], x[i], s);
        h1[o] = fmaxf(s, 0.f);
    }
#pragma unroll 4
    for (int o = 0; o < H; ++o) {
        float s = w[OB2 + o];
#pragma unroll 8
        for (int i = 0; i < H; ++i) s = fmaf(w[OW2 + o * H + i], h1[i], s);
        h2[o] = fmaxf(s, 0.f);
    }
#pragma unroll
    for (int o = 0; o < DOUT; ++o) {
        float s = w[OB3 + o];
#pragma unroll 8
        for (int i = 0; i < H; ++i) s = fmaf(w[OW3 + o * H + i], h2[i], s);
        y[o] = s;
    }
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float *__restrict__ wg, int rows, const float *__restrict__ X,
                                                     float *__restrict__ Y) {
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = wg[i];
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float x[DIN], h1[H], h2[H], y[DOUT];
#pragma unroll
    for (int i = 0; i < DIN; ++i) x[i] = X[(long long)r * DIN + i];
    forward_row(w, x, h1, h2, y);
#pragma unroll
    for (int o = 0; o < DOUT; ++o) Y[(long long)r * DOUT + o] = y[o];
}

// Per-tile partial gradient (unscaled: dL/dy = 2 m (y - t)) and partial
// loss numerator / mask sum.
struct TileBuf {
    float x[TILE][DIN];
    float h1[TILE][H + 1];
    float h2[TILE][H + 1];
    float d1[TILE][H + 1];
    float d2[TILE][H + 1];
    float dy[TILE][DOUT];
    float red[2][TILE];
};

__global__ void __launch_bounds__(TILE) k_mlp_tile_grad(const float *__restrict__ wg, int rows, const float *__restrict__ X,
                                                        const float *__restrict__ T, const float *__restrict__ M,
                                                        float *__restrict__ part) {
    extern __shared__ float smem[];
    float *w = smem;
    TileBuf &tb = *reinterpret_cast<TileBuf *>(smem + NP + (4 - NP % 4) % 4);
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = wg[i];
    __syncthreads();
    const int t = threadIdx.x;
    const int r = blockIdx.x * TILE + t;
    const bool live = r < rows;
    float x[DIN], h1[H], h2[H], y[DOUT];
#pragma unroll
    for (int i = 0; i < DIN; ++i) x[i] = live ? X[(long long)r * DIN + i] : 0.f;
    forward_row(w, x, h1, h2, y);
    float lnum = 0.f, msum = 0.f;
    float dy[DOUT];
#pragma unroll
    for (int o = 0; o < DOUT; ++o) {
        const float m = live ? M[(long long)r * DOUT + o] : 0.f;
        const float e = live ? y[o] - T[(long long)r * DOUT + o] : 0.f;
        lnum = fmaf(m * e, e, lnum);
        msum += m;
        dy[o] = 2.f * m * e;
    }
    float d2[H];
#pragma unroll 4
    for (int i = 0; i < H; ++i) {
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < DOUT; ++o) s = fmaf(w[OW3 + o * H + i], dy[o], s);
        d2[i] = h2[i] > 0.f ? s : 0.f;
    }
#pragma unroll 4
    for (int i = 0; i < H; ++i) {
        float s = 0.f;
#pragma unroll 8
        for (int o = 0; o < H; ++o) s = fmaf(w[OW2 + o * H + i], d2[o], s);
        tb.d1[t][i] = h1[i] > 0.f ? s : 0.f;
    }
#pragma unroll
    for (int i = 0; i < DIN; ++i) tb.x[t][i] = x[i];
#pragma unroll
    for (int i = 0; i < H; ++i) { tb.h1[t][i] = h1[i]; tb.h2[t][i] = h2[i]; tb.d2[t][i] = d2[i]; }
#pragma unroll
    for (int o = 0; o < DOUT; ++o) tb.dy[t][o] = dy[o];
    tb.red[0][t] = lnum;
    tb.red[1][t] = msum;
    __syncthreads();
    // weight-gradient entries of this tile: sum over the tile's rows
    float *out = part + (long long)blockIdx.x * (NP + 2);
    for (int e = t; e < NP; e += blockDim.x) {
        float s = 0.f;
        if (e < OB1) {
            const int o = e / DIN, i = e - o * DIN;
            for (int q = 0; q < TILE; ++q) s = fmaf(tb.d1[q][o], tb.x[q][i], s);
        } else if (e < OW2) {
            const int o = e - OB1;
            for (int q = 0; q < TILE; ++q) s += tb.d1[q][o];
        } else if (e < OB2) {
            const int o = (e - OW2) / H, i = (e - OW2) - o * H;
            for (int q = 0; q < TILE; ++q) s = fmaf(tb.d2[q][o], tb.h1[q][i], s);
        } else if (e < OW3) {
            const int o = e - OB2;
            for (int q = 0; q < TILE; ++q) s += tb.d2[q][o];
        } else if (e < OB3) {
            const int o = (e - OW3) / H, i = (e - OW3) - o * H;
            for (int q = 0; q < TILE; ++q) s = fmaf(tb.dy[q][o], tb.h2[q][i], s);
        } else {
            const int o = e - OB3;
            for (int q = 0; q < TILE; ++q) s += tb.dy[q][o];
        }
        out[e] = s;
    }
    if (t < 2) {
        float s = 0.f;
        for (int q = 0; q < TILE; ++q) s += tb.red[t][q];
        out[NP + t] = s;
    }
}

// grad[e] = sum_tiles part[tile][e] / max(1, sum mask); loss likewise.
__global__ void k_mlp_reduce(const float *__restrict__ part, int tiles, float *__restrict__ grad, float *__restrict__ loss) {
    float msum = 0.f;
    for (int q = 0; q < tiles; ++q) msum += part[(long long)q * (NP + 2) + NP + 1];
    const float denom = fmaxf(msum, 1.f);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e <= NP) {
        float s = 0.f;
        for (int q = 0; q < tiles; ++q) s += part[(long long)q * (NP + 2) + e];
        if (e < NP) grad[e] = s / denom;
        else *loss = s / denom;
    }
}

// One Adam step (Kingma & Ba, Algorithm 1) with bias correction at step t.
__global__ void k_adam(int np, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

size_t tile_smem() { return (size_t)(NP + (4 - NP % 4) % 4) * 4 + sizeof(TileBuf); }

}  // namespace

size_t mlp_workspace(int rows) {
    const size_t tiles = (size_t)ceil_div(rows, TILE);
    return ((tiles * (NP + 2) * 4 + 255) / 256) * 256;
}

cudaError_t launch_mlp_forward(int din, const float *w, int rows, const float *X, float *Y, cudaStream_t st) {
    if (din != DIN) return cudaErrorNotSupported;
    k_mlp_forward<<<ceil_div(rows, 128), 128, 0, st>>>(w, rows, X, Y);
    return cudaPeekAtLastError();
}

cudaError_t launch_mlp_loss_grad(int din, const float *w, int rows, const float *X, const float *T, const float *M,
                                 float *grad, float *loss, void *ws, cudaStream_t st) {
    if (din != DIN) return cudaErrorNotSupported;
    const int tiles = ceil_div(rows, TILE);
    const size_t sm = tile_smem();
    cudaError_t e = prepare(k_mlp_tile_grad, sm);
    if (e != cudaSuccess) return e;
    float *part = static_cast<float *>(ws);
    k_mlp_tile_grad<<<tiles, TILE, sm, st>>>(w, rows, X, T, M, part);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return e;
    k_mlp_reduce<<<ceil_div(NP + 1, 256), 256, 0, st>>>(part, tiles, grad, loss);
    return cudaPeekAtLastError();
}

cudaError_t launch_mlp_adam(int np, float *w, const float *g, float *m, float *v, int t, float lr, float b1, float b2,
                            float eps, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<ceil_div(np, 256), 256, 0, st>>>(np, w, g, m, v, lr, b1, b2, eps, c1, c2);
    return cudaPeekAtLastError();
}

}  // namespace glass
