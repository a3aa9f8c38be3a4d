// dev_umma.cuh -- fifth-generation tensor cores (tcgen05 "UMMA") for the
// batched order-64 GEMM: C = A B with FP32 operands through a TF32 split
// (a = a_hi + a_lo, a_hi = tf32(a), a_lo = tf32(a - a_hi); the product sums
// a_x b_y over x, y in {hi, lo}), FP32 accumulation in tensor memory.
//
// One persistent CTA per SM walks problems p = blockIdx.x,
// blockIdx.x + gridDim.x, ... through a pipeline of three warp roles:
//   - the issue warp has the bulk-copy engine (cp.async.bulk, completion on
//     an mbarrier) bring problem i + 2's A and B (16 KB each, contiguous)
//     into raw[i % 2], and issues problem i's 8 tcgen05.mma (one per K = 8
//     step, M = N = 128 over the stacked hi / lo operands) into one of the
//     tensor-memory accumulators;
//   - the split warps turn problem i's raw operands into stacked hi / lo
//     tiles in the K-major 128-byte-swizzled layout in op[i % 2];
//   - the drain warps move finished accumulators (tcgen05.ld) to HBM.
// Every wait is bounded (about a second of clock cycles); on a timeout the
// CTA records the failure in a device status word, stops issuing work,
// waits (bounded again) for what it has in flight, frees its tensor memory
// and returns.
#pragma once

#include "common.cuh"

namespace glass {
namespace umma {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// --------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Wait until the phase of parity `parity` has completed; false after about
// `cycles` clock cycles without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long cycles) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > cycles) return false;
    }
}

// ------------------------------------------------------------ bulk copies
// Global -> shared, `bytes` (multiple of 16, both addresses 16-byte aligned),
// completion counted on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Generic-proxy shared-memory writes become visible to the async proxy
// (tensor cores, bulk copies).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------- tensor memory
template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t *slot) {  // one whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(NCOLS)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOLS>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {  // the allocating warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(NCOLS) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit columns of this thread's lane (shape 32x32b: warp
// w % 4 reads lanes 32 (w % 4) .. +31), waited for before returning.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = __uint_as_float(r[u]);
}

// 32 consecutive columns, likewise.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = __uint_as_float(r[u]);
}

// ---------------------------------------------------------- descriptors
// Shared-memory matrix descriptor, K-major without swizzling: start address,
// leading-dimension byte offset (between core matrices adjacent along K),
// stride byte offset (between adjacent 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, no negation, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A B over one K = 8 step, operands from shared memory.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The mbarrier receives one arrival once every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// ----------------------------------------------------------- 3xTF32 tiles
// a = hi + lo: hi = a rounded to TF32 (11 significant bits, ties away from
// zero: add half a TF32 unit to the bit pattern and clear the 13 low bits,
// on the integer pipe), lo = a - hi (exact), rounded the same way.
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split4(const float (&x)[4], float4 &hi, float4 &lo) {
    float h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        h[u] = tf32_round(x[u]);
        l[u] = tf32_round(x[u] - h[u]);
    }
    hi = make_float4(h[0], h[1], h[2], h[3]);
    lo = make_float4(l[0], l[1], l[2], l[3]);
}

// Operand tiles: K-major with the 128-byte swizzle, hi and lo stacked into
// one 128-row operand per matrix (rows 0-63 the hi parts, 64-127 the lo
// parts of rows / columns 0-63).  Element (r, k) of the stacked operand
// (r = row of A or column of B, c4 = k / 4 its 16-byte chunk) lies in K-half
// k / 32 (16 KB each), row r at 128 r bytes, chunk c4 % 8 at chunk position
// (c4 % 8) ^ (r % 8).  8-row groups are 1024 B apart (SBO); the K = 8 step s
// starts 32 (s % 4) bytes into the rows of half s / 4, and the hardware
// applies the same XOR to the addresses it forms (the tiles sit on 1 KB
// boundaries).
constexpr int TILE_FLOATS = 64 * 64;     // one raw 64 x 64 operand
constexpr int PAIR_FLOATS = 2 * TILE_FLOATS;  // one stacked hi / lo operand

__device__ __forceinline__ int pair_off(int r, int c4) {  // r < 64: the hi part; + 2048 floats: the lo part
    return (c4 >> 3) * 4096 + r * 32 + (((c4 & 7) ^ (r & 7)) << 2);
}
__device__ __forceinline__ uint64_t kstep_desc(uint32_t pair, int s) {
    return desc_kmajor(pair + (s >> 2) * 16384 + (s & 3) * 32, 16, 1024) | (2ull << 61);
}

// A (column-major, pitch 64), T threads: thread t splits row
// m = t % 32 + 32 ((t / 32) % 2) at k-chunks c4 = t / 64 + (T / 64) it: four
// scalar loads per chunk (consecutive m across a warp), and the eight rows
// of a quarter-warp store to eight distinct chunk positions.
template <int T>
__device__ __forceinline__ void split_a(const float *raw, float *pair, int t) {
    const int w = t >> 5, m = (t & 31) + 32 * (w & 1);
#pragma unroll
    for (int it = 0; it < 1024 / T; ++it) {
        const int c4 = (w >> 1) + (T / 64) * it;
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = raw[(4 * c4 + u) * 64 + m];
        float4 h, l;
        split4(x, h, l);
        const int o = pair_off(m, c4);
        *reinterpret_cast<float4 *>(pair + o) = h;
        *reinterpret_cast<float4 *>(pair + o + 2048) = l;
    }
}

// B (column-major K x N, pitch 64: K contiguous), T threads: thread t
// handles column n = 8 rg + q (q = t % 8) at chunk c4 with
// c4 % 8 = alpha(q) ^ (j % 8), alpha = multiplication by a primitive element
// of GF(8) (x^3 + x + 1): over a quarter-warp (q = 0..7) both the loaded
// chunk positions alpha(q) ^ j and the stored ones alpha(q) ^ q ^ j are all
// distinct, so neither side has bank conflicts.
__device__ __forceinline__ int gf8_alpha(int q) { return ((q << 1) & 7) ^ ((q & 4) ? 3 : 0); }

template <int T>
__device__ __forceinline__ void split_b(const float *raw, float *pair, int t) {
    const int q = t & 7, grp = t >> 3;
#pragma unroll
    for (int it = 0; it < 1024 / T; ++it) {
        const int lin = grp + (T / 8) * it, rg = lin & 7, j = lin >> 3;
        const int c4 = (j & 8) | (gf8_alpha(q) ^ (j & 7)), n = 8 * rg + q;
        const float4 v = *reinterpret_cast<const float4 *>(raw + n * 64 + 4 * c4);
        const float x[4] = {v.x, v.y, v.z, v.w};
        float4 h, l;
        split4(x, h, l);
        const int o = pair_off(n, c4);
        *reinterpret_cast<float4 *>(pair + o) = h;
        *reinterpret_cast<float4 *>(pair + o + 2048) = l;
    }
}

// One product: per k-step a single M = N = 128 MMA of the stacked operands
// forms all four products a_x b_y (x, y in {hi, lo}) in the quadrants of the
// accumulator -- lane = row of the stacked A, columns d .. d + 127 = the
// columns of the stacked B -- so C is the sum of the four quadrants (the
// lo * lo quadrant comes at no extra cost).
__device__ __forceinline__ void issue_split_product(uint32_t d, const float *ap, const float *bp) {
    constexpr uint32_t ID = idesc_tf32(128, 128);
    const uint32_t a = smem_u32(ap), b = smem_u32(bp);
#pragma unroll
    for (int s = 0; s < 8; ++s) mma_tf32(d, kstep_desc(a, s), kstep_desc(b, s), ID, s > 0 ? 1u : 0u);
}

// ------------------------------------------------------- pipelined kernel
constexpr int RAW_BYTES = 2 * TILE_FLOATS * 4;  // A and B of one problem
constexpr int OP_BYTES = 2 * PAIR_FLOATS * 4;   // stacked A and B of one problem
constexpr int BAR_OFF = 2 * RAW_BYTES + 2 * OP_BYTES;
// The drain warps exchange half sums through two 64 x 65 buffers (pitch 65:
// conflict-free along rows and columns).
constexpr int XCH_OFF = BAR_OFF + 256, XCH_FLOATS = 64 * 65;
// Two raw stages, two operand stages (1 KB aligned), the mbarriers, the
// tensor-memory slot and the failure flag, the exchange buffers.
constexpr int SMEM_BYTES = XCH_OFF + 2 * XCH_FLOATS * 4;
constexpr long long WAIT_CYCLES = 2000000000LL;  // about a second
// Values of the CTA's failure flag: a bounded wait gave up, or the dynamic
// shared memory is not 1 KB aligned (the swizzled tiles cannot be placed).
constexpr int kFailTimeout = 1, kFailUnaligned = 2;

// C[p] = A[p] B[p] for p = blockIdx.x, blockIdx.x + gridDim.x, ... < batch;
// every operand 64 x 64, contiguous (batch stride 4096 floats), 16-byte
// aligned.  Warp-specialised: SW split warps (4 or 8), four drain warps
// (drain warp w reads lane quarter w % 4), one issue warp (bulk copies and
// MMAs, lane 0); AS accumulators of 128 columns in tensor memory (2 or 4).
// The roles meet only on mbarriers (problem i of the CTA; s = i % 2,
// a = i % AS):
//   raw_full[s]  bulk copy of problem i landed in raw[s]      (tx bytes)
//   op_full[s]   split of problem i written to op[s]          (SW * 32 arrivals)
//   mma_done[a]  MMAs of problem i complete: op[s] reusable, accumulator a readable
//   acc_free[a]  accumulator a drained                        (128 arrivals)
// each waited on with the parity of its use count (i / 2 or i / AS), and the
// drain warps meet on named barrier 1 for the half-sum exchange.  Every
// wait gives up after wait_cycles clock cycles; *status then gets
// GLASS_ERR_TIMEOUT (GLASS_ERR_UNSUPPORTED if the shared memory could not be
// aligned), every later wait is skipped, nothing new is issued and C is not
// written, so every role still reaches its barriers.  withhold_loads != 0
// (a test of that path) makes the issue warp start no bulk copy at all, so
// the first waits run out with nothing in flight.
template <int SW, int AS>
__global__ void __launch_bounds__(32 * (SW + 5), 1)
    k_gemm_umma64(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C, int batch,
                  unsigned *status, long long wait_cycles, int withhold_loads) {
    static_assert((SW == 4 || SW == 8) && (AS == 2 || AS == 4), "warp roles, accumulator stages");
    constexpr int TCOLS = AS * 128;  // a power of two
    extern __shared__ __align__(1024) unsigned char smem[];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    float *raw = reinterpret_cast<float *>(smem);
    float *op = reinterpret_cast<float *>(smem + 2 * RAW_BYTES);
    uint64_t *raw_full = reinterpret_cast<uint64_t *>(smem + BAR_OFF);
    uint64_t *op_full = raw_full + 2, *mma_done = op_full + 2, *acc_free = mma_done + AS;
    uint32_t *slot = reinterpret_cast<uint32_t *>(acc_free + AS);
    volatile int *failed = reinterpret_cast<volatile int *>(slot + 1);

    const int G = gridDim.x, first = blockIdx.x;
    const int count = first < batch ? (batch - first + G - 1) / G : 0;
    if (t == 0) {
        *failed = (smem_u32(op) & 1023u) != 0 ? kFailUnaligned : 0;  // the swizzle atoms need 1 KB alignment
        for (int k = 0; k < 2; ++k) {
            mbar_init(&raw_full[k], 1);
            mbar_init(&op_full[k], SW * 32);
        }
        for (int k = 0; k < AS; ++k) {
            mbar_init(&mma_done[k], 1);
            mbar_init(&acc_free[k], 128);
        }
        fence_mbar_init();
    }
    __syncwarp();
    if (w == 0) {
        tmem_alloc<TCOLS>(slot);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *slot;

    auto wait = [&](uint64_t *bar, int use) {
        if (*failed) return;
        if (!mbar_wait(bar, use & 1, wait_cycles)) *failed = kFailTimeout;
    };
    auto prob = [&](int i) { return (first + (long long)i * G) * TILE_FLOATS; };

    if (w < SW) {
        // ---- split warps
        for (int i = 0; i < count; ++i) {
            const int s = i & 1;
            wait(&raw_full[s], i >> 1);
            if (i >= 2) wait(&mma_done[(i - 2) % AS], (i - 2) / AS);  // problem i - 2 has left op[s]
            const float *r = raw + s * 2 * TILE_FLOATS;
            float *o = op + s * 2 * PAIR_FLOATS;
            split_a<SW * 32>(r, o, t);
            split_b<SW * 32>(r + TILE_FLOATS, o + PAIR_FLOATS, t);
            fence_async_smem();
            mbar_arrive(&op_full[s]);
        }
    } else if (w < SW + 4) {
        // ---- drain warps: lane quarter q holds rows 32 (q % 2) + lane of the
        // a_hi (q < 2) or a_lo (q >= 2) half; each sums its two column halves,
        // quarters 2, 3 hand theirs to 0, 1, which store whole 128-byte
        // column segments of C
        const int q = w & 3, r = 32 * (q & 1) + lane;
        float *xch = reinterpret_cast<float *>(smem + XCH_OFF);
        for (int i = 0; i < count; ++i) {
            const int a = i % AS;
            wait(&mma_done[a], i / AS);
            fence_after_sync();
            const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + 128 * a;
            float hold[64];
#pragma unroll
            for (int cc = 0; cc < 64; cc += 32) {
                float v[32], v2[32];
                tmem_ld32(ta + cc, v);
                tmem_ld32(ta + 64 + cc, v2);
#pragma unroll
                for (int u = 0; u < 32; ++u) hold[cc + u] = v[u] + v2[u];
            }
            fence_before_sync();
            mbar_arrive(&acc_free[a]);
            float *xb = xch + (i & 1) * XCH_FLOATS;
            if (q >= 2)
#pragma unroll
                for (int u = 0; u < 64; ++u) xb[r * 65 + u] = hold[u];
            asm volatile("bar.sync 1, 128;" ::: "memory");
            float *c = C + prob(i);
            if (q < 2 && !*failed)  // after a failure the accumulator holds no product: C stays untouched
#pragma unroll
                for (int u = 0; u < 64; ++u) __stcs(c + u * 64 + r, hold[u] + xb[r * 65 + u]);
        }
    } else if (lane == 0) {
        // ---- issue warp
        int issued = 0, loaded = 0;
        auto load = [&](int i) {
            float *dst = raw + (i & 1) * 2 * TILE_FLOATS;
            mbar_expect_tx(&raw_full[i & 1], 2 * TILE_FLOATS * 4);
            bulk_g2s(dst, A + prob(i), TILE_FLOATS * 4, &raw_full[i & 1]);
            bulk_g2s(dst + TILE_FLOATS, B + prob(i), TILE_FLOATS * 4, &raw_full[i & 1]);
            loaded = i + 1;
        };
        for (int i = 0; i < 2 && i < count && !*failed && !withhold_loads; ++i) load(i);
        for (int i = 0; i < count; ++i) {
            const int s = i & 1, a = i % AS;
            wait(&op_full[s], i >> 1);  // split done: raw[s] consumed, op[s] ready
            if (*failed) break;
            if (i + 2 < count && !withhold_loads) load(i + 2);
            if (i >= AS) wait(&acc_free[a], i / AS - 1);  // problem i - AS drained from accumulator a
            if (*failed) break;
            fence_after_sync();
            const float *o = op + s * 2 * PAIR_FLOATS;
            issue_split_product(tbase + 128 * a, o, o + PAIR_FLOATS);
            mma_commit(&mma_done[a]);
            issued = i + 1;
        }
        if (*failed) {
            // bounded waits for what is still in flight: the last MMA groups
            // committed and the bulk copies not yet consumed
            for (int k = issued - 1; k >= 0 && k >= issued - 2; --k)
                mbar_wait(&mma_done[k % AS], (k / AS) & 1, WAIT_CYCLES);
            for (int k = loaded - 1; k >= 0 && k >= loaded - 2; --k)
                mbar_wait(&raw_full[k & 1], (k >> 1) & 1, WAIT_CYCLES);
            atomicExch(status, *failed == kFailUnaligned ? (unsigned)GLASS_ERR_UNSUPPORTED
                                                         : (unsigned)GLASS_ERR_TIMEOUT);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (w == 0) {
        fence_after_sync();
        tmem_dealloc<TCOLS>(tbase);
    }
}

// ------------------------------------------------------------- BF16 mode
// C = A B with BF16 operands (stored as bf16, column-major 64 x 64) and FP32
// accumulation: no split; one K-major 128-byte-swizzled 64-row tile per
// operand (a row is one 128-byte swizzle atom: element (r, k) at byte
// 128 r + 16 ((k / 8) ^ (r % 8)) + 2 (k % 8)) and four tcgen05.mma of
// kind::f16 (M = N = 64, K = 16) per product.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

constexpr int BF_TILE_BYTES = 64 * 128;  // one 64 x 64 bf16 operand

__device__ __forceinline__ int bf_off(int r, int c) {  // bytes; c = k / 8, the 16-byte chunk
    return r * 128 + ((c ^ (r & 7)) << 4);
}

// A (column-major bf16, pitch 64): thread t builds row m = t % 64, chunks
// c = t / 64 + (T / 64) it from eight 2-byte loads (consecutive m across a
// warp); a quarter-warp's eight rows store to eight distinct chunk positions.
template <int T>
__device__ __forceinline__ void bf16_tile_a(const unsigned short *raw, unsigned char *tile, int t) {
    const int m = t & 63;
#pragma unroll
    for (int it = 0; it < 512 / T; ++it) {
        const int c = (t >> 6) + (T / 64) * it;
        unsigned short h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) h[u] = raw[(8 * c + u) * 64 + m];
        uint4 v;
        v.x = h[0] | ((unsigned)h[1] << 16);
        v.y = h[2] | ((unsigned)h[3] << 16);
        v.z = h[4] | ((unsigned)h[5] << 16);
        v.w = h[6] | ((unsigned)h[7] << 16);
        *reinterpret_cast<uint4 *>(tile + bf_off(m, c)) = v;
    }
}

// B (column-major K x N bf16: a column is one 128-byte row of the K-major
// tile): each 16-byte chunk moves to its swizzled position; chunk choice
// alpha(q) ^ j as in split_b keeps loads and stores conflict free.
template <int T>
__device__ __forceinline__ void bf16_tile_b(const unsigned char *raw, unsigned char *tile, int t) {
    const int q = t & 7, grp = t >> 3;
#pragma unroll
    for (int it = 0; it < 512 / T; ++it) {
        const int lin = grp + (T / 8) * it, rg = lin & 7, j = lin >> 3;  // j < 8
        const int c = gf8_alpha(q) ^ j, n = 8 * rg + q;
        *reinterpret_cast<uint4 *>(tile + bf_off(n, c)) = *reinterpret_cast<const uint4 *>(raw + n * 128 + c * 16);
    }
}

constexpr int BF_RAW_BYTES = 2 * BF_TILE_BYTES;  // A and B of one problem, as stored
constexpr int BF_OP_BYTES = 2 * BF_TILE_BYTES;   // the two swizzled tiles
constexpr int BF_BAR_OFF = 2 * BF_RAW_BYTES + 2 * BF_OP_BYTES;
constexpr int BF_SMEM_BYTES = BF_BAR_OFF + 256;

// Same pipeline and failure handling as k_gemm_umma64 (two raw and two tile
// stages, AS = 2 accumulators of 64 columns; four tile warps, four drain
// warps -- lanes 0-15 of each lane quarter hold rows 16 q .. 16 q + 15 of an
// M = 64 accumulator -- and one issue warp); small enough for two CTAs per
// SM.
__global__ void __launch_bounds__(288, 2)
    k_gemm_umma64_bf16(const unsigned short *__restrict__ A, const unsigned short *__restrict__ B,
                       float *__restrict__ C, int batch, unsigned *status, long long wait_cycles) {
    constexpr int SW = 4, AS = 2, TCOLS = 128;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    unsigned char *raw = smem;
    unsigned char *op = smem + 2 * BF_RAW_BYTES;
    uint64_t *raw_full = reinterpret_cast<uint64_t *>(smem + BF_BAR_OFF);
    uint64_t *op_full = raw_full + 2, *mma_done = op_full + 2, *acc_free = mma_done + AS;
    uint32_t *slot = reinterpret_cast<uint32_t *>(acc_free + AS);
    volatile int *failed = reinterpret_cast<volatile int *>(slot + 1);

    const int G = gridDim.x, first = blockIdx.x;
    const int count = first < batch ? (batch - first + G - 1) / G : 0;
    if (t == 0) {
        *failed = (smem_u32(op) & 1023u) != 0 ? kFailUnaligned : 0;
        for (int k = 0; k < 2; ++k) {
            mbar_init(&raw_full[k], 1);
            mbar_init(&op_full[k], SW * 32);
        }
        for (int k = 0; k < AS; ++k) {
            mbar_init(&mma_done[k], 1);
            mbar_init(&acc_free[k], 128);
        }
        fence_mbar_init();
    }
    __syncwarp();
    if (w == 0) {
        tmem_alloc<TCOLS>(slot);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *slot;

    auto wait = [&](uint64_t *bar, int use) {
        if (*failed) return;
        if (!mbar_wait(bar, use & 1, wait_cycles)) *failed = kFailTimeout;
    };
    auto prob = [&](int i) { return (first + (long long)i * G) * TILE_FLOATS; };  // elements

    if (w < SW) {
        for (int i = 0; i < count; ++i) {
            const int s = i & 1;
            wait(&raw_full[s], i >> 1);
            if (i >= 2) wait(&mma_done[(i - 2) % AS], (i - 2) / AS);
            const unsigned char *r = raw + s * BF_RAW_BYTES;
            unsigned char *o = op + s * BF_OP_BYTES;
            bf16_tile_a<SW * 32>(reinterpret_cast<const unsigned short *>(r), o, t);
            bf16_tile_b<SW * 32>(r + BF_TILE_BYTES, o + BF_TILE_BYTES, t);
            fence_async_smem();
            mbar_arrive(&op_full[s]);
        }
    } else if (w < SW + 4) {
        const int q = w & 3, row = lane < 16 ? 16 * q + lane : -1;
        for (int i = 0; i < count; ++i) {
            const int a = i % AS;
            wait(&mma_done[a], i / AS);
            fence_after_sync();
            const uint32_t ta = tbase + ((uint32_t)(32 * q) << 16) + 64 * a;
            float *c = C + prob(i);
#pragma unroll
            for (int cc = 0; cc < 64; cc += 32) {
                float v[32];
                tmem_ld32(ta + cc, v);
                if (row >= 0 && !*failed)
#pragma unroll
                    for (int u = 0; u < 32; ++u) __stcs(c + (cc + u) * 64 + row, v[u]);
            }
            fence_before_sync();
            mbar_arrive(&acc_free[a]);
        }
    } else if (lane == 0) {
        int issued = 0, loaded = 0;
        auto load = [&](int i) {
            unsigned char *dst = raw + (i & 1) * BF_RAW_BYTES;
            mbar_expect_tx(&raw_full[i & 1], BF_RAW_BYTES);
            bulk_g2s(dst, A + prob(i), BF_TILE_BYTES, &raw_full[i & 1]);
            bulk_g2s(dst + BF_TILE_BYTES, B + prob(i), BF_TILE_BYTES, &raw_full[i & 1]);
            loaded = i + 1;
        };
        for (int i = 0; i < 2 && i < count && !*failed; ++i) load(i);
        for (int i = 0; i < count; ++i) {
            const int s = i & 1, a = i % AS;
            wait(&op_full[s], i >> 1);
            if (*failed) break;
            if (i + 2 < count) load(i + 2);
            if (i >= AS) wait(&acc_free[a], i / AS - 1);
            if (*failed) break;
            fence_after_sync();
            const uint32_t ta = smem_u32(op + s * BF_OP_BYTES), tb = ta + BF_TILE_BYTES;
            constexpr uint32_t ID = idesc_bf16(64, 64);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_f16(tbase + 64 * a, desc_kmajor(ta + 32 * k, 16, 1024) | (2ull << 61),
                        desc_kmajor(tb + 32 * k, 16, 1024) | (2ull << 61), ID, k > 0 ? 1u : 0u);
            mma_commit(&mma_done[a]);
            issued = i + 1;
        }
        if (*failed) {
            for (int k = issued - 1; k >= 0 && k >= issued - 2; --k)
                mbar_wait(&mma_done[k % AS], (k / AS) & 1, WAIT_CYCLES);
            for (int k = loaded - 1; k >= 0 && k >= loaded - 2; --k)
                mbar_wait(&raw_full[k & 1], (k >> 1) & 1, WAIT_CYCLES);
            atomicExch(status, *failed == kFailUnaligned ? (unsigned)GLASS_ERR_UNSUPPORTED
                                                         : (unsigned)GLASS_ERR_TIMEOUT);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (w == 0) {
        fence_after_sync();
        tmem_dealloc<TCOLS>(tbase);
    }
}

}  // namespace umma
}  // namespace glass
