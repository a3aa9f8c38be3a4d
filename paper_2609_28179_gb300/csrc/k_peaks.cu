// k_peaks.cu -- pipe-throughput probes: kernels that keep one arithmetic
// pipe busy with independent work and a known operation count, timed by the
// caller to obtain the measured peak a roofline is quoted against (FP32
// FFMA, FP64 DFMA, and the mma.sync shapes the library's tensor-core paths
// use: TF32 m16n8k8 and BF16 m16n8k16).
#include <cstdint>

#include "common.cuh"
#include "glass.h"

namespace glass {
namespace {

constexpr int kChains = 8;  // independent accumulators per thread

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T seed, T *sink) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T x = (T)0.999, y = (T)0.001;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-1) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the work
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_mma_probe(int iters, float *sink) {
    const unsigned lane = threadIdx.x & 31;
    // small values (bit patterns of ~1e-3 in either format) keep the sums finite
    const unsigned av = BF16 ? 0x3a833a83u : 0x3a830000u;
    unsigned a[4] = {av ^ lane, av, av, av ^ (lane << 1)}, b[2] = {av, av ^ lane};
    float d[kChains][4];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) d[c][r] = 0.f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (BF16) mma_bf16(d[c], a, b);
            else mma_tf32(d[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace glass

using namespace glass;

extern "C" glass_status glass_peak_probe(int kind, int iters, int blocks, int threads, void *sink, double *flops,
                                         glass_stream_t stream) {
    if (kind < 0 || kind > 3 || iters < 1 || blocks < 1 || threads < 32 || threads > 256 || (threads & 31) ||
        sink == nullptr)
        return GLASS_ERR_INVALID_VALUE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double th = (double)blocks * threads;
    double f = 0.0;
    switch (kind) {
        case 0:
            k_fma_probe<float><<<blocks, threads, 0, st>>>(iters, 1.f, static_cast<float *>(sink));
            f = th * iters * 8.0 * kChains * 2.0;
            break;
        case 1:
            k_fma_probe<double><<<blocks, threads, 0, st>>>(iters, 1.0, static_cast<double *>(sink));
            f = th * iters * 8.0 * kChains * 2.0;
            break;
        case 2:
            k_mma_probe<false><<<blocks, threads, 0, st>>>(iters, static_cast<float *>(sink));
            f = th / 32.0 * iters * kChains * (2.0 * 16 * 8 * 8);
            break;
        default:
            k_mma_probe<true><<<blocks, threads, 0, st>>>(iters, static_cast<float *>(sink));
            f = th / 32.0 * iters * kChains * (2.0 * 16 * 8 * 16);
            break;
    }
    if (flops != nullptr) *flops = f;
    return cudaPeekAtLastError() == cudaSuccess ? GLASS_OK : GLASS_ERR_CUDA;
}
