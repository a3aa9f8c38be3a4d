// k_gemm_tc.cu -- batched tensor-core GEMM C = A B for n in {16, 32, 64}
// with FP32 accumulation: BF16 operands, TF32 operands, or 3xTF32 split
// products (a = a_hi + a_lo with a_hi = tf32(a), a_lo = tf32(a - a_hi);
// C += a_lo b_hi + a_hi b_lo + a_hi b_hi), the precision path the paper
// lists as future work (Sec. V).  The BF16 and 3xTF32 products of order 64
// run on the fifth-generation tensor cores (dev_umma.cuh), which also serve
// the FP32 block-scope GEMM of order 64; the others use warp-level mma.sync.
//
// Work split: n/16 warps per product, warp w owns rows 16w .. 16w+15 of C
// and every 8-column block, so one A fragment serves n/8 MMAs.  A CTA holds
// 4 warps (4/(n/16) products); orders 16 to 32 (TF32 modes) and 16, 32
// (BF16) run a persistent streaming form instead (one warp per product,
// the next product prefetched).  Operands are staged into shared memory with
// coalesced 16-byte streaming loads, in padded layouts whose leading
// dimensions make every fragment load bank-conflict free; C goes back
// through shared memory for coalesced 16-byte stores.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "dev_umma.cuh"

namespace glass {
namespace {

__device__ __forceinline__ unsigned tf32_rna(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int N>
struct TcShape {
    static constexpr int WP = N / 16;        // warps per product
    static constexpr int PPC = 4 / WP;       // products per CTA
    static constexpr int NB = N / 8;         // 8-column blocks
    static constexpr int LDC = N + 4;        // C staging (floats)
};

// ------------------------------------------------------------------ TF32
// As: A column-major, lda = N + 8 floats; Bs: B column-major, ldb = N + 4.
template <int N, bool SPLIT>
__global__ void __launch_bounds__(128) k_gemm_tf32(const float *__restrict__ A, const float *__restrict__ B,
                                                   float *__restrict__ C, int batch) {
    using S = TcShape<N>;
    constexpr int LDA = N + 8, LDB = N + 4;
    constexpr int PER = N * LDA + N * LDB;
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lp = warp / S::WP, wq = warp % S::WP;  // product in CTA, warp within product
    const int b0 = blockIdx.x * S::PPC;
    // stage all products of the CTA (float4, coalesced)
    for (int p = 0; p < S::PPC; ++p) {
        const int b = b0 + p;
        if (b >= batch) break;
        float *As = smem + p * PER, *Bs = As + N * LDA;
        const float4 *ga = reinterpret_cast<const float4 *>(A + (long long)b * N * N);
        const float4 *gb = reinterpret_cast<const float4 *>(B + (long long)b * N * N);
        for (int v = threadIdx.x; v < N * N / 4; v += blockDim.x) {
            const int col = (4 * v) / N, row = (4 * v) % N;
            *reinterpret_cast<float4 *>(As + col * LDA + row) = __ldcs(ga + v);
            *reinterpret_cast<float4 *>(Bs + col * LDB + row) = __ldcs(gb + v);
        }
    }
    __syncthreads();
    const int b = b0 + lp;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = 16 * wq;
    float acc[S::NB][4];
#pragma unroll
    for (int j = 0; j < S::NB; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const float *As = smem + lp * PER, *Bs = As + N * LDA;
    if (b < batch) {
#pragma unroll 2
        for (int k0 = 0; k0 < N; k0 += 8) {
            float af[4];
            af[0] = As[(k0 + t) * LDA + m0 + g];
            af[1] = As[(k0 + t) * LDA + m0 + g + 8];
            af[2] = As[(k0 + t + 4) * LDA + m0 + g];
            af[3] = As[(k0 + t + 4) * LDA + m0 + g + 8];
            unsigned ah[4], al[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ah[u] = tf32_rna(af[u]);
                if (SPLIT) al[u] = tf32_rna(af[u] - __uint_as_float(ah[u]));
            }
#pragma unroll
            for (int j = 0; j < S::NB; ++j) {
                const float b0v = Bs[(8 * j + g) * LDB + k0 + t], b1v = Bs[(8 * j + g) * LDB + k0 + t + 4];
                unsigned bh[2] = {tf32_rna(b0v), tf32_rna(b1v)};
                if (SPLIT) {
                    unsigned bl[2] = {tf32_rna(b0v - __uint_as_float(bh[0])), tf32_rna(b1v - __uint_as_float(bh[1]))};
                    mma_tf32(acc[j], al, bh);
                    mma_tf32(acc[j], ah, bl);
                }
                mma_tf32(acc[j], ah, bh);
            }
        }
    }
    __syncthreads();
    // C fragments -> shared (column-major, ld LDC) -> global
    float *Cs = smem + lp * (N * S::LDC);
    if (b < batch) {
#pragma unroll
        for (int j = 0; j < S::NB; ++j) {
            const int c0 = 8 * j + 2 * t;
            Cs[c0 * S::LDC + m0 + g] = acc[j][0];
            Cs[(c0 + 1) * S::LDC + m0 + g] = acc[j][1];
            Cs[c0 * S::LDC + m0 + g + 8] = acc[j][2];
            Cs[(c0 + 1) * S::LDC + m0 + g + 8] = acc[j][3];
        }
    }
    __syncthreads();
    for (int p = 0; p < S::PPC; ++p) {
        const int bb = b0 + p;
        if (bb >= batch) break;
        const float *cs = smem + p * (N * S::LDC);
        float4 *gc = reinterpret_cast<float4 *>(C + (long long)bb * N * N);
        for (int v = threadIdx.x; v < N * N / 4; v += blockDim.x) {
            const int col = (4 * v) / N, row = (4 * v) % N;
            __stcs(gc + v, *reinterpret_cast<const float4 *>(cs + col * S::LDC + row));
        }
    }
}

// ------------------------------------------------ TF32, orders 16 .. 32
// Persistent streaming form for n in {16, 24, 32} (one warp per product;
// 3 n^2 floats of HBM traffic against 2 n^3 flops: a stream, not a
// contraction): each warp walks the batch with a stride of the grid's warp
// count; the next product's A and B are copied by cp.async into the warp's
// second buffer while the current one is multiplied, so no barrier stands
// between a load and its use.  C leaves straight from the accumulator
// fragments (lanes g = 0..7 of a fragment row cover one 32-byte column
// segment: whole sectors).  Row tiles are 16 high: at n = 24 the second one
// reads rows 24..31 of A's padding, zeroed once, and its rows past n are not
// stored.
template <int N>
struct Stream {
    static constexpr int LDA = N == 24 ? 40 : N + 8;  // 8 mod 32: conflict-free A fragments
    static constexpr int LDB = N + 4;                 // 4 mod 8: conflict-free B fragments
    static constexpr int MT = (N + 15) / 16, NT = N / 8;
    static constexpr int BUF = N * LDA + N * LDB;     // floats per buffer
    static constexpr int WARPS = N == 32 ? 2 : 8;     // warps per CTA
    static constexpr int CTAS = N == 24 ? 2 : 5;      // resident CTAs per SM (shared memory)
    static constexpr size_t SMEM = (size_t)WARPS * 2 * BUF * 4;
};

template <int N, bool SPLIT>
__global__ void __launch_bounds__(32 * Stream<N>::WARPS) k_gemm_tf32_stream(const float *__restrict__ A,
                                                                          const float *__restrict__ B,
                                                                          float *__restrict__ C, int batch) {
    using S = Stream<N>;
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float *buf = smem + warp * 2 * S::BUF;
    const int stride = gridDim.x * S::WARPS;  // <= CTAS * SMs * WARPS
    int b = blockIdx.x * S::WARPS + warp;
    if (b >= batch) return;  // whole warp
    if (N == 24) {           // rows 24..31 of both A buffers are read as zero
        for (int e = lane; e < 2 * N * 8; e += 32) {
            const int h = e / (N * 8), c = (e / 8) % N, r = 24 + e % 8;
            buf[h * S::BUF + c * S::LDA + r] = 0.f;
        }
    }
    auto issue = [&](int bb, float *dst) {
        const float *ga = A + (long long)bb * N * N, *gb = B + (long long)bb * N * N;
        float *As = dst, *Bs = dst + N * S::LDA;
#pragma unroll
        for (int e = lane; e < N * N / 4; e += 32) {
            const int c = e / (N / 4), r = 4 * (e % (N / 4));
            cp_async16(As + c * S::LDA + r, ga + c * N + r);
            cp_async16(Bs + c * S::LDB + r, gb + c * N + r);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(b, buf);
    for (int it = 0; b < batch; ++it) {
        float *cur = buf + (it & 1) * S::BUF;
        const int nb = b < batch - stride ? b + stride : batch;  // no int overflow near 2^31
        if (nb < batch) {
            issue(nb, buf + ((it + 1) & 1) * S::BUF);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        const float *As = cur, *Bs = cur + N * S::LDA;
        float acc[S::MT][S::NT][4];
#pragma unroll
        for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < S::NT; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
#pragma unroll
        for (int k0 = 0; k0 < N; k0 += 8) {
            unsigned ah[S::MT][4], al[S::MT][4];
#pragma unroll
            for (int mt = 0; mt < S::MT; ++mt) {
                const float af[4] = {As[(k0 + t) * S::LDA + 16 * mt + g], As[(k0 + t) * S::LDA + 16 * mt + g + 8],
                                     As[(k0 + t + 4) * S::LDA + 16 * mt + g],
                                     As[(k0 + t + 4) * S::LDA + 16 * mt + g + 8]};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    ah[mt][u] = tf32_rna(af[u]);
                    if (SPLIT) al[mt][u] = tf32_rna(af[u] - __uint_as_float(ah[mt][u]));
                }
            }
#pragma unroll
            for (int nt = 0; nt < S::NT; ++nt) {
                const float b0v = Bs[(8 * nt + g) * S::LDB + k0 + t], b1v = Bs[(8 * nt + g) * S::LDB + k0 + t + 4];
                unsigned bh[2] = {tf32_rna(b0v), tf32_rna(b1v)};
                unsigned bl[2] = {0u, 0u};
                if (SPLIT) {
                    bl[0] = tf32_rna(b0v - __uint_as_float(bh[0]));
                    bl[1] = tf32_rna(b1v - __uint_as_float(bh[1]));
                }
#pragma unroll
                for (int mt = 0; mt < S::MT; ++mt) {
                    if (SPLIT) {
                        mma_tf32(acc[mt][nt], al[mt], bh);
                        mma_tf32(acc[mt][nt], ah[mt], bl);
                    }
                    mma_tf32(acc[mt][nt], ah[mt], bh);
                }
            }
        }
        __syncwarp();  // the buffer is refilled two products on
        float *gc = C + (long long)b * N * N;
#pragma unroll
        for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < S::NT; ++nt) {
                const int c = 8 * nt + 2 * t, r = 16 * mt + g;
                __stcs(gc + c * N + r, acc[mt][nt][0]);
                __stcs(gc + (c + 1) * N + r, acc[mt][nt][1]);
                if (r + 8 < N) {
                    __stcs(gc + c * N + r + 8, acc[mt][nt][2]);
                    __stcs(gc + (c + 1) * N + r + 8, acc[mt][nt][3]);
                }
            }
        b = nb;
    }
}

// ------------------------------------------------- BF16, orders 16 and 32
// The streaming form of the BF16 product (as k_gemm_tf32_stream: one warp
// per product, the next product's operands copied by cp.async into the
// warp's second buffer while the current one multiplies, C written from
// the accumulator fragments).  A stays column-major in shared memory as
// copied; ldmatrix.trans forms its row-major m16n8k16 fragments (pairs
// along k) from four 8 x 8 sub-blocks, and B's column-major pairs are
// single 32-bit loads.  Pitch N + 8 halves: the eight 16-byte rows of every
// ldmatrix sub-block and the B fragments fall in distinct banks.
template <int N>
struct StreamBf {
    static constexpr int LD = N + 8;                  // halves per column
    static constexpr int MT = N / 16, NT = N / 8;
    static constexpr int BUF = 2 * N * LD;            // halves per buffer (A, then B)
    static constexpr int WARPS = 8;
    static constexpr int CTAS = N == 16 ? 8 : 2;      // resident CTAs per SM (shared memory)
    static constexpr size_t SMEM = (size_t)WARPS * 2 * BUF * 2;
};

__device__ __forceinline__ void ldmatrix_x4_trans(unsigned (&r)[4], const void *smem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

template <int N>
__global__ void __launch_bounds__(32 * StreamBf<N>::WARPS) k_gemm_bf16_stream(const __nv_bfloat16 *__restrict__ A,
                                                                            const __nv_bfloat16 *__restrict__ B,
                                                                            float *__restrict__ C, int batch) {
    using S = StreamBf<N>;
    extern __shared__ __align__(16) unsigned short hsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    unsigned short *buf = hsm + warp * 2 * S::BUF;
    const int stride = gridDim.x * S::WARPS;  // <= CTAS * SMs * WARPS
    int b = blockIdx.x * S::WARPS + warp;
    if (b >= batch) return;  // whole warp
    auto issue = [&](int bb, unsigned short *dst) {
        const __nv_bfloat16 *ga = A + (long long)bb * N * N, *gb = B + (long long)bb * N * N;
#pragma unroll
        for (int e = lane; e < N * N / 8; e += 32) {  // 16-byte chunks: 8 halves of one column
            const int c = e / (N / 8), r = 8 * (e % (N / 8));
            cp_async16(dst + c * S::LD + r, ga + c * N + r);
            cp_async16(dst + N * S::LD + c * S::LD + r, gb + c * N + r);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // this lane's ldmatrix row: sub-block lane / 8 (rows +8 for odd, k +8 for the upper two)
    const int lr = lane & 7, lm = lane >> 3;
    const int a_row = 8 * (lm & 1), a_k = lr + 8 * (lm >> 1);
    issue(b, buf);
    for (int it = 0; b < batch; ++it) {
        unsigned short *cur = buf + (it & 1) * S::BUF;
        const int nb = b < batch - stride ? b + stride : batch;  // no int overflow near 2^31
        if (nb < batch) {
            issue(nb, buf + ((it + 1) & 1) * S::BUF);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        const unsigned short *As = cur, *Bs = cur + N * S::LD;
        float acc[S::MT][S::NT][4];
#pragma unroll
        for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < S::NT; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
#pragma unroll
        for (int k0 = 0; k0 < N; k0 += 16) {
            unsigned a[S::MT][4];
#pragma unroll
            for (int mt = 0; mt < S::MT; ++mt) ldmatrix_x4_trans(a[mt], As + (k0 + a_k) * S::LD + 16 * mt + a_row);
#pragma unroll
            for (int nt = 0; nt < S::NT; ++nt) {
                unsigned bq[2];
                bq[0] = *reinterpret_cast<const unsigned *>(Bs + (8 * nt + g) * S::LD + k0 + 2 * t);
                bq[1] = *reinterpret_cast<const unsigned *>(Bs + (8 * nt + g) * S::LD + k0 + 2 * t + 8);
#pragma unroll
                for (int mt = 0; mt < S::MT; ++mt) mma_bf16(acc[mt][nt], a[mt], bq);
            }
        }
        __syncwarp();  // the buffer is refilled two products on
        float *gc = C + (long long)b * N * N;
#pragma unroll
        for (int mt = 0; mt < S::MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < S::NT; ++nt) {
                const int c = 8 * nt + 2 * t, r = 16 * mt + g;
                __stcs(gc + c * N + r, acc[mt][nt][0]);
                __stcs(gc + (c + 1) * N + r, acc[mt][nt][1]);
                __stcs(gc + c * N + r + 8, acc[mt][nt][2]);
                __stcs(gc + (c + 1) * N + r + 8, acc[mt][nt][3]);
            }
        b = nb;
    }
}


}  // namespace

cudaError_t launch_gemm_umma64_ex(const float *A, const float *B, float *C, int batch, long long wait_cycles,
                                  int withhold_loads, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    if (((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15) != 0)
        return cudaErrorInvalidConfiguration;
    unsigned *status = device_status_word();
    if (status == nullptr) return cudaErrorInvalidDeviceFunction;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    constexpr int kSplitWarps = 8, kAccumulators = 2;  // measured best of {4, 8} x {2, 4}
    auto kern = umma::k_gemm_umma64<kSplitWarps, kAccumulators>;
    if ((e = prepare(kern, umma::SMEM_BYTES)) != cudaSuccess) return e;
    kern<<<batch < sms ? batch : sms, 32 * (kSplitWarps + 5), umma::SMEM_BYTES, st>>>(A, B, C, batch, status,
                                                                                       wait_cycles, withhold_loads);
    return cudaPeekAtLastError();
}

cudaError_t launch_gemm_umma64(const float *A, const float *B, float *C, int batch, cudaStream_t st) {
    return launch_gemm_umma64_ex(A, B, C, batch, umma::WAIT_CYCLES, 0, st);
}

// BF16 products of order 64 on the fifth-generation tensor cores (kind::f16).
cudaError_t launch_gemm_umma64_bf16(const void *A, const void *B, float *C, int batch, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    // 8 KB bulk copies of A and B, 16-byte stores of C
    if (((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15) != 0)
        return cudaErrorInvalidConfiguration;
    unsigned *status = device_status_word();
    if (status == nullptr) return cudaErrorInvalidDeviceFunction;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if ((e = prepare(umma::k_gemm_umma64_bf16, umma::BF_SMEM_BYTES)) != cudaSuccess) return e;
    const int grid = batch < 2 * sms ? batch : 2 * sms;  // two CTAs per SM
    umma::k_gemm_umma64_bf16<<<grid, 288, umma::BF_SMEM_BYTES, st>>>(static_cast<const unsigned short *>(A),
                                                                     static_cast<const unsigned short *>(B), C,
                                                                     batch, status, umma::WAIT_CYCLES);
    return cudaPeekAtLastError();
}

// The streaming TF32 kernels of orders 16, 24 and 32: a grid of resident
// CTAs whose warps stride over the batch.  Operands packed (ld = n, stride
// n^2) and 16-byte aligned, as launch_gemm_tc requires.
cudaError_t launch_gemm_tf32_stream(int n, bool split, const float *A, const float *B, float *C, int batch,
                                    cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
#define TS(NN, SP) do { using S = Stream<NN>;                                                              \
        if ((e = prepare(k_gemm_tf32_stream<NN, SP>, S::SMEM)) != cudaSuccess) return e;                    \
        const int grid = std::min(ceil_div(batch, S::WARPS), S::CTAS * sms);                                \
        k_gemm_tf32_stream<NN, SP><<<grid, 32 * S::WARPS, S::SMEM, st>>>(A, B, C, batch);                    \
        return cudaPeekAtLastError(); } while (0)
    if (n == 16) { if (split) TS(16, true); TS(16, false); }
    if (n == 24) { if (split) TS(24, true); TS(24, false); }
    if (n == 32) { if (split) TS(32, true); TS(32, false); }
#undef TS
    return cudaErrorInvalidConfiguration;
}

cudaError_t launch_gemm_tc(int n, int math, const void *A, const void *B, float *C, int batch, cudaStream_t st) {
    // 16-byte staging needs 16-byte aligned operands
    if (((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15) != 0)
        return cudaErrorInvalidConfiguration;
    const int ppc = 4 / (n / 16);
    const int grid = ceil_div(batch, ppc);
    cudaError_t e;
    if (math == GLASS_MATH_BF16_TC) {
        const __nv_bfloat16 *a = static_cast<const __nv_bfloat16 *>(A), *b = static_cast<const __nv_bfloat16 *>(B);
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
#define BF(NN) do { using S = StreamBf<NN>;                                                               \
        if ((e = prepare(k_gemm_bf16_stream<NN>, S::SMEM)) != cudaSuccess) return e;                       \
        const int gs = std::min(ceil_div(batch, S::WARPS), S::CTAS * sms);                                  \
        k_gemm_bf16_stream<NN><<<gs, 32 * S::WARPS, S::SMEM, st>>>(a, b, C, batch);                         \
        return cudaPeekAtLastError(); } while (0)
        if (n == 16) BF(16);
        if (n == 32) BF(32);
#undef BF
        return launch_gemm_umma64_bf16(A, B, C, batch, st);
    }
    const size_t smem = (size_t)ppc * (n * (n + 8) + n * (n + 4)) * 4;
    const float *a = static_cast<const float *>(A), *b = static_cast<const float *>(B);
#define TF(NN, SP) do { if ((e = prepare(k_gemm_tf32<NN, SP>, smem)) != cudaSuccess) return e;           \
        k_gemm_tf32<NN, SP><<<grid, 128, smem, st>>>(a, b, C, batch); return cudaPeekAtLastError(); } while (0)
    if (n <= 32) return launch_gemm_tf32_stream(n, math == GLASS_MATH_3XTF32_TC, a, b, C, batch, st);
    if (math == GLASS_MATH_TF32_TC) TF(64, false);
    return launch_gemm_umma64(a, b, C, batch, st);
#undef TF
}

}  // namespace glass
