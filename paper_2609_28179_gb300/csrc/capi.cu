// capi.cu -- the library's C ABI: argument validation, placement
// resolution and dispatch to the batched kernels.  See include/glass.h for
// the contract of every entry point.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "placement_table.h"
#include "riccati_table.h"
#include "robo_table.h"
#include "fp64_table.h"

namespace glass {

cudaError_t prepare_kernel(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, fn);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}

// Device status word (bounded waits that gave up, ...), one per device.
__device__ unsigned g_device_status;

unsigned *device_status_word() {
    unsigned *p = nullptr;
    return cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_device_status) == cudaSuccess ? p : nullptr;
}

namespace {

const glass_opts kDefaultOpts = {GLASS_F32, GLASS_MATH_FP32, GLASS_LAYOUT_COLMAJOR, {GLASS_SCOPE_AUTO, 0}, 0, 0, 0,
                                  GLASS_RESIDUAL_FP64};

const glass_opts &opts_or_default(const glass_opts *o) { return o ? *o : kDefaultOpts; }

glass_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return GLASS_OK;
    if (e == cudaErrorInvalidConfiguration) return GLASS_ERR_INVALID_VALUE;
    if (e == cudaErrorNotSupported) return GLASS_ERR_UNSUPPORTED;
    return GLASS_ERR_CUDA;
}

bool valid_pack(int p) { return p == 1 || p == 2 || p == 4 || p == 8; }

Mat make_mat(const void *p, int ld, long long s, int rows, int cols, int layout) {
    Mat m;
    m.p = const_cast<float *>(static_cast<const float *>(p));
    m.ld = ld;
    m.s = s;
    m.rows = rows;
    m.cols = cols;
    m.layout = layout;
    if (layout == GLASS_LAYOUT_INTERLEAVED32) {
        m.ld = rows;
        m.s = (long long)rows * cols;
    }
    return m;
}

// Checks of one column-major operand: ld >= rows and, for an output, a batch
// stride that keeps problems disjoint (inputs may share storage, s == 0).
bool operand_ok(const void *p, int ld, long long s, int rows, int cols, bool output, int layout) {
    if (p == nullptr) return false;
    if (layout == GLASS_LAYOUT_INTERLEAVED32) return true;
    if (ld < rows || s < 0) return false;
    if (output && s < (long long)ld * (cols - 1) + rows) return false;
    return true;
}

bool feasible(int op, int n, int k, Placement pl) {
    switch (op) {
        case GLASS_OP_GEMM: return feasible_gemm(n, n, k, pl);
        case GLASS_OP_POSV:
        case GLASS_OP_POTRF:
        case GLASS_OP_POTRS:
        case GLASS_OP_TRSM: return feasible_chol(op, n, k, pl);
        case GLASS_OP_GETRF_GETRS: return feasible_lu(n, k, pl);
        case GLASS_OP_ROT3: return feasible_geom(0, k, pl);
        case GLASS_OP_SE3: return feasible_geom(1, k, pl);
        default: return false;
    }
}

// ------------------------------------------------------- learned model
struct Learned {
    bool set = false;
    float w[5516];
    float mean[8], stdv[8];
};
Learned g_learned;
std::mutex g_learned_mu;

// Row of the placement table / output index of the cost model.
int table_op(int op) {
    switch (op) {
        case GLASS_OP_POTRF:
        case GLASS_OP_POTRS: return GLASS_OP_POSV;
        default: return op;
    }
}

// Model index of a matrix op (gemm, posv, trsm, getrf_getrs) or -1.
int model_op(int op) {
    switch (table_op(op)) {
        case GLASS_OP_GEMM: return 0;
        case GLASS_OP_POSV: return 1;
        case GLASS_OP_TRSM: return 2;
        case GLASS_OP_GETRF_GETRS: return 3;
        default: return -1;
    }
}

void learned_predict(const Learned &L, const float x[8], float y[12]) {
    const float *W1 = L.w, *b1 = W1 + 64 * 8, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64, *b3 = W3 + 12 * 64;
    float h1[64], h2[64];
    for (int o = 0; o < 64; ++o) {
        float s = b1[o];
        for (int i = 0; i < 8; ++i) s += W1[o * 8 + i] * x[i];
        h1[o] = s > 0.f ? s : 0.f;
    }
    for (int o = 0; o < 64; ++o) {
        float s = b2[o];
        for (int i = 0; i < 64; ++i) s += W2[o * 64 + i] * h1[i];
        h2[o] = s > 0.f ? s : 0.f;
    }
    for (int o = 0; o < 12; ++o) {
        float s = b3[o];
        for (int i = 0; i < 64; ++i) s += W3[o * 64 + i] * h2[i];
        y[o] = s;
    }
}

bool on_grid(int op, int n, int batch) {
    (void)op;
    bool gn = false, gb = false;
    for (int i = 0; i < kTableNumN; ++i) gn |= kTableN[i] == n;
    for (int i = 0; i < kTableNumB; ++i) gb |= kTableB[i] == batch;
    return gn && gb;
}

int nearest_index(const int *grid, int cnt, double v) {
    int best = 0;
    double bd = 1e300;
    for (int i = 0; i < cnt; ++i) {
        const double d = fabs(log2((double)grid[i]) - log2(v));
        if (d < bd - 1e-12) { bd = d; best = i; }
    }
    return best;
}

Placement decode(unsigned char code) { return Placement{code >> 2, 1 << (code & 3)}; }

Placement resolve(int op, int n, int k, int batch, int use_learned) {
    const int top = table_op(op);
    if (use_learned && model_op(op) >= 0 && !on_grid(op, n, batch)) {
        std::lock_guard<std::mutex> lk(g_learned_mu);
        if (g_learned.set) {
            float x[8] = {0, 0, 0, 0, (float)log2((double)n), (float)log2((double)(k > 0 ? k : 1)),
                          (float)log2((double)(batch > 0 ? batch : 1)), 0.f};
            x[model_op(op)] = 1.f;
            for (int i = 0; i < 8; ++i) x[i] = (x[i] - g_learned.mean[i]) / g_learned.stdv[i];
            float y[12];
            learned_predict(g_learned, x, y);
            int best = -1;
            for (int p = 0; p < 12; ++p) {
                const Placement pl = decode((unsigned char)p);
                if (!feasible(op, n, k, pl)) continue;
                if (best < 0 || y[p] < y[best]) best = p;
            }
            if (best >= 0) return decode((unsigned char)best);
        }
    }
    const int ni = nearest_index(kTableN, kTableNumN, (top == GLASS_OP_ROT3 || top == GLASS_OP_SE3) ? k : n);
    const int bi = nearest_index(kTableB, kTableNumB, batch > 0 ? batch : 1);
    Placement pl = decode(kTable[top][ni][bi]);
    if (feasible(op, n, k, pl)) return pl;
    // nearest feasible: widen the scope, keep the pack if possible
    for (int s = pl.scope; s <= SCOPE_BLOCK; ++s)
        for (int pk = pl.pack; pk >= 1; pk >>= 1) {
            const Placement q{s, pk};
            if (feasible(op, n, k, q)) return q;
        }
    return Placement{SCOPE_WARP, 1};
}

// Placement of a call: explicit (validated) or resolved from the table.
// The interleaved layout is served at thread scope only.
glass_status placement_of(int op, int n, int k, int batch, const glass_opts &o, Placement &pl) {
    const bool inter = o.layout == GLASS_LAYOUT_INTERLEAVED32;
    if (o.placement.scope == GLASS_SCOPE_AUTO) {
        pl = resolve(op, n, k, batch, o.use_learned);
        if (inter && pl.scope != SCOPE_THREAD) pl = Placement{SCOPE_THREAD, 1};
        if (o.placement.pack != 0) {
            if (!valid_pack(o.placement.pack)) return GLASS_ERR_INVALID_VALUE;
            pl.pack = o.placement.pack;
        }
    } else {
        if (o.placement.scope < GLASS_SCOPE_THREAD || o.placement.scope > GLASS_SCOPE_BLOCK)
            return GLASS_ERR_INVALID_VALUE;
        pl.scope = o.placement.scope;
        pl.pack = o.placement.pack == 0 ? 1 : o.placement.pack;
        if (!valid_pack(pl.pack)) return GLASS_ERR_INVALID_VALUE;
    }
    if (inter && pl.scope != SCOPE_THREAD) return GLASS_ERR_UNSUPPORTED;
    if (!feasible(op, n, k, pl)) return inter ? GLASS_ERR_UNSUPPORTED : GLASS_ERR_INVALID_VALUE;
    return GLASS_OK;
}

glass_status check_common(const glass_opts &o) {
    if (o.layout != GLASS_LAYOUT_COLMAJOR && o.layout != GLASS_LAYOUT_INTERLEAVED32) return GLASS_ERR_INVALID_VALUE;
    if (o.dtype != GLASS_F32 && o.dtype != GLASS_F64 && o.dtype != GLASS_BF16) return GLASS_ERR_INVALID_VALUE;
    if (o.math < GLASS_MATH_FP32 || o.math > GLASS_MATH_3XTF32_TC) return GLASS_ERR_INVALID_VALUE;
    return GLASS_OK;
}

glass_status check_order(int n) {
    if (n < 1) return GLASS_ERR_INVALID_VALUE;
    if (n > 64) return GLASS_ERR_UNSUPPORTED;
    return GLASS_OK;
}

// ------------------------------------------------------ FP64 storage
int f64_row(int op) {
    switch (op) {
        case GLASS_OP_GEMM: return 0;
        case GLASS_OP_POSV:
        case GLASS_OP_POTRF:
        case GLASS_OP_POTRS: return 1;
        case GLASS_OP_TRSM: return 2;
        default: return 3;
    }
}

glass_status f64_placement_of(int op, int n, int batch, const glass_opts &o, Placement &pl) {
    if (o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR) return GLASS_ERR_UNSUPPORTED;
    if (o.placement.scope == GLASS_SCOPE_AUTO) {
        const int ni = nearest_index(kF64N, kF64NumN, n);
        const int bi = nearest_index(kF64B, kF64NumB, batch > 0 ? batch : 1);
        pl = decode(kF64Table[f64_row(op)][ni][bi]);
        if (o.placement.pack != 0) {
            if (!valid_pack(o.placement.pack)) return GLASS_ERR_INVALID_VALUE;
            pl.pack = o.placement.pack;
        }
        if (!feasible_f64(op, n, pl)) {
            pl.scope = SCOPE_WARP;
            while (!feasible_f64(op, n, pl) && pl.pack > 1) pl.pack >>= 1;
        }
    } else {
        pl = Placement{o.placement.scope, o.placement.pack == 0 ? 1 : o.placement.pack};
        if (!valid_pack(pl.pack)) return GLASS_ERR_INVALID_VALUE;
    }
    return feasible_f64(op, n, pl) ? GLASS_OK : GLASS_ERR_INVALID_VALUE;
}

// ------------------------------------------------- robotics operations
Placement robo_resolve(int op, int n, int batch) {
    const int bi = nearest_index(kRoboB, kRoboNumB, batch > 0 ? batch : 1);
    const Placement pl = decode(kRoboTable[op][bi]);
    if (feasible_robo(op, n, pl)) return pl;
    return Placement{SCOPE_THREAD, 1};
}

glass_status robo_placement_of(int op, int n, int batch, const glass_opts &o, Placement &pl) {
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    if (o.placement.scope == GLASS_SCOPE_AUTO) {
        pl = robo_resolve(op, n, batch);
        if (o.placement.pack != 0) {
            if (!valid_pack(o.placement.pack)) return GLASS_ERR_INVALID_VALUE;
            pl.pack = o.placement.pack;
        }
    } else {
        pl = Placement{o.placement.scope, o.placement.pack == 0 ? 1 : o.placement.pack};
    }
    return feasible_robo(op, n, pl) ? GLASS_OK : GLASS_ERR_INVALID_VALUE;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// ------------------------------------------------------- LQR gain placement
constexpr int kComposedCode = 12;

size_t ric_workspace(int nx, int nu, int batch) {
    const size_t pb = ((size_t)batch * nx * nu + 63) / 64 * 64;
    return (pb + (size_t)batch * nu * nu) * 4;
}

Placement ric_fused_fallback(int nx, int nu, Placement want) {
    for (int s = want.scope; s <= SCOPE_BLOCK; ++s)
        for (int pk = want.pack; pk >= 1; pk >>= 1) {
            const Placement q{s, pk};
            if (feasible_riccati(nx, nu, q)) return q;
        }
    return Placement{SCOPE_BLOCK, 1};
}

Placement ric_resolve(int nx, int nu, int batch, bool composed_ok) {
    int best = 0;
    double bd = 1e300;
    for (int i = 0; i < kRicNum; ++i) {
        const double d = fabs(log2((double)kRicNx[i]) - log2((double)nx)) + fabs(log2((double)kRicNu[i]) - log2((double)nu));
        if (d < bd - 1e-12) { bd = d; best = i; }
    }
    const int bi = nearest_index(kRicB, kRicNumB, batch > 0 ? batch : 1);
    const unsigned char code = kRicTable[best][bi];
    if (code == kComposedCode) {
        if (composed_ok) return Placement{GLASS_SCOPE_COMPOSED, 1};
        return ric_fused_fallback(nx, nu, Placement{SCOPE_WARP, 1});
    }
    const Placement pl = decode(code);
    if (feasible_riccati(nx, nu, pl)) return pl;
    const Placement q = ric_fused_fallback(nx, nu, pl);
    if (!feasible_riccati(nx, nu, q) && composed_ok) return Placement{GLASS_SCOPE_COMPOSED, 1};
    return q;
}

}  // namespace
}  // namespace glass

using namespace glass;

#define GLASS_TRY(x) do { glass_status _s = (x); if (_s != GLASS_OK) return _s; } while (0)

extern "C" {

glass_status glass_batched_gemm(int m, int n, int k, const void *A, int lda, long long sA, const void *B, int ldb,
                                long long sB, void *C, int ldc, long long sC, int batch, const glass_opts *opts,
                                glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (m < 1 || n < 1 || k < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (m > 64 || n > 64 || k > 64) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (o.math != GLASS_MATH_FP32) {
        if (!(m == n && n == k && (n == 16 || n == 32 || n == 64))) return GLASS_ERR_UNSUPPORTED;
        if (o.layout != GLASS_LAYOUT_COLMAJOR) return GLASS_ERR_UNSUPPORTED;
        if (o.math == GLASS_MATH_BF16_TC && o.dtype != GLASS_BF16) return GLASS_ERR_INVALID_VALUE;
        if (o.math != GLASS_MATH_BF16_TC && o.dtype != GLASS_F32) return GLASS_ERR_INVALID_VALUE;
        if (!A || !B || !C) return GLASS_ERR_INVALID_VALUE;
        if (lda != n || ldb != n || ldc != n || sA != (long long)n * n || sB != (long long)n * n ||
            sC != (long long)n * n)
            return GLASS_ERR_UNSUPPORTED;
        return from_cuda(launch_gemm_tc(n, o.math, A, B, static_cast<float *>(C), batch, st));
    }
    if (o.dtype == GLASS_F64) {
        if (!operand_ok(A, lda, sA, m, k, false, o.layout) || !operand_ok(B, ldb, sB, k, n, false, o.layout) ||
            !operand_ok(C, ldc, sC, m, n, true, o.layout))
            return GLASS_ERR_INVALID_VALUE;
        const int mx = m > n ? (m > k ? m : k) : (n > k ? n : k);
        Placement pl;
        GLASS_TRY(f64_placement_of(GLASS_OP_GEMM, mx, batch, o, pl));
        return from_cuda(launch_gemm_f64(m, n, k, static_cast<const double *>(A), lda, sA,
                                         static_cast<const double *>(B), ldb, sB, static_cast<double *>(C), ldc, sC,
                                         batch, pl, st));
    }
    if (o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!operand_ok(A, lda, sA, m, k, false, o.layout) || !operand_ok(B, ldb, sB, k, n, false, o.layout) ||
        !operand_ok(C, ldc, sC, m, n, true, o.layout))
        return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    const int nn = m > n ? (m > k ? m : k) : (n > k ? n : k);
    if (o.placement.scope == GLASS_SCOPE_AUTO && o.layout == GLASS_LAYOUT_COLMAJOR) {
        pl = resolve(GLASS_OP_GEMM, nn, nn, batch, o.use_learned);
        if (o.placement.pack != 0) pl.pack = o.placement.pack;
        if (!feasible_gemm(m, n, k, pl)) {
            pl = Placement{SCOPE_WARP, 1};
            if (!feasible_gemm(m, n, k, pl)) pl = Placement{SCOPE_BLOCK, 1};
        }
    } else {
        GLASS_TRY(placement_of(GLASS_OP_GEMM, nn, nn, batch, o, pl));
    }
    if (o.layout == GLASS_LAYOUT_INTERLEAVED32 && pl.scope != SCOPE_THREAD) return GLASS_ERR_UNSUPPORTED;
    if (!feasible_gemm(m, n, k, pl)) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_gemm(m, n, k, make_mat(A, lda, sA, m, k, o.layout), make_mat(B, ldb, sB, k, n, o.layout),
                                 make_mat(C, ldc, sC, m, n, o.layout), batch, pl, st));
}

glass_status glass_batched_potrf(int n, void *A, int lda, long long sA, int *info, int batch, const glass_opts *opts,
                                 glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    GLASS_TRY(check_order(n));
    if (batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (batch == 0) return GLASS_OK;
    if (o.dtype == GLASS_F64) {
        if (!operand_ok(A, lda, sA, n, n, true, o.layout) || info == nullptr) return GLASS_ERR_INVALID_VALUE;
        Placement pl;
        GLASS_TRY(f64_placement_of(GLASS_OP_POTRF, n, batch, o, pl));
        return from_cuda(launch_chol_f64(GLASS_OP_POTRF, n, 0, static_cast<double *>(A), lda, sA, nullptr, 1, 0, info,
                                         batch, pl, reinterpret_cast<cudaStream_t>(stream)));
    }
    if (o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!operand_ok(A, lda, sA, n, n, true, o.layout) || info == nullptr) return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    GLASS_TRY(placement_of(GLASS_OP_POTRF, n, 1, batch, o, pl));
    return from_cuda(launch_potrf(n, make_mat(A, lda, sA, n, n, o.layout), info, batch, pl,
                                  o.fp64_diag ? NUM_FP64_DIAG : 0, reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_potrs(int n, int nrhs, const void *L, int lda, long long sA, void *B, int ldb, long long sB,
                                 int batch, const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    GLASS_TRY(check_order(n));
    if (nrhs < 0 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (batch == 0 || nrhs == 0) return GLASS_OK;
    if (o.dtype == GLASS_F64) {
        if (!operand_ok(L, lda, sA, n, n, false, o.layout) || !operand_ok(B, ldb, sB, n, nrhs, true, o.layout))
            return GLASS_ERR_INVALID_VALUE;
        Placement pl;
        GLASS_TRY(f64_placement_of(GLASS_OP_POTRS, n, batch, o, pl));
        return from_cuda(launch_chol_f64(GLASS_OP_POTRS, n, nrhs, static_cast<double *>(const_cast<void *>(L)), lda,
                                         sA, static_cast<double *>(B), ldb, sB, nullptr, batch, pl,
                                         reinterpret_cast<cudaStream_t>(stream)));
    }
    if (o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!operand_ok(L, lda, sA, n, n, false, o.layout) || !operand_ok(B, ldb, sB, n, nrhs, true, o.layout))
        return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    GLASS_TRY(placement_of(GLASS_OP_POTRS, n, nrhs, batch, o, pl));
    return from_cuda(launch_potrs(n, nrhs, make_mat(L, lda, sA, n, n, o.layout),
                                  make_mat(B, ldb, sB, n, nrhs, o.layout), batch, pl,
                                  reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_posv(int n, int nrhs, void *A, int lda, long long sA, void *B, int ldb, long long sB,
                                int *info, int batch, const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    GLASS_TRY(check_order(n));
    if (nrhs < 0 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (o.refine_steps < 0 || o.refine_steps > 1) return GLASS_ERR_UNSUPPORTED;
    if (o.residual != GLASS_RESIDUAL_FP64 && o.residual != GLASS_RESIDUAL_DOT2) return GLASS_ERR_INVALID_VALUE;
    if (batch == 0) return GLASS_OK;
    if (o.dtype == GLASS_F64) {
        if (o.refine_steps != 0) return GLASS_ERR_UNSUPPORTED;
        if (!operand_ok(A, lda, sA, n, n, true, o.layout) || info == nullptr) return GLASS_ERR_INVALID_VALUE;
        if (nrhs > 0 && !operand_ok(B, ldb, sB, n, nrhs, true, o.layout)) return GLASS_ERR_INVALID_VALUE;
        Placement pl;
        GLASS_TRY(f64_placement_of(GLASS_OP_POSV, n, batch, o, pl));
        return from_cuda(launch_chol_f64(nrhs > 0 ? GLASS_OP_POSV : GLASS_OP_POTRF, n, nrhs, static_cast<double *>(A),
                                         lda, sA, static_cast<double *>(B), ldb, sB, info, batch, pl,
                                         reinterpret_cast<cudaStream_t>(stream)));
    }
    if (o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!operand_ok(A, lda, sA, n, n, true, o.layout) || info == nullptr) return GLASS_ERR_INVALID_VALUE;
    if (nrhs > 0 && !operand_ok(B, ldb, sB, n, nrhs, true, o.layout)) return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    GLASS_TRY(placement_of(GLASS_OP_POSV, n, nrhs > 0 ? nrhs : 1, batch, o, pl));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (nrhs == 0)
        return from_cuda(launch_potrf(n, make_mat(A, lda, sA, n, n, o.layout), info, batch, pl,
                                      o.fp64_diag ? NUM_FP64_DIAG : 0, st));
    const int num = (o.fp64_diag ? NUM_FP64_DIAG : 0) | (o.residual == GLASS_RESIDUAL_DOT2 ? NUM_DOT2_RESIDUAL : 0);
    return from_cuda(launch_posv(n, nrhs, make_mat(A, lda, sA, n, n, o.layout), make_mat(B, ldb, sB, n, nrhs, o.layout),
                                 info, batch, pl, num, o.refine_steps, st));
}

glass_status glass_batched_trsm(int n, int nrhs, const void *L, int lda, long long sA, void *B, int ldb, long long sB,
                                int batch, const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    GLASS_TRY(check_order(n));
    if (nrhs < 0 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (nrhs > 4096) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0 || nrhs == 0) return GLASS_OK;
    if (o.dtype == GLASS_F64) {
        if (!operand_ok(L, lda, sA, n, n, false, o.layout) || !operand_ok(B, ldb, sB, n, nrhs, true, o.layout))
            return GLASS_ERR_INVALID_VALUE;
        Placement pl;
        GLASS_TRY(f64_placement_of(GLASS_OP_TRSM, n, batch, o, pl));
        return from_cuda(launch_chol_f64(GLASS_OP_TRSM, n, nrhs, static_cast<double *>(const_cast<void *>(L)), lda,
                                         sA, static_cast<double *>(B), ldb, sB, nullptr, batch, pl,
                                         reinterpret_cast<cudaStream_t>(stream)));
    }
    if (o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!operand_ok(L, lda, sA, n, n, false, o.layout) || !operand_ok(B, ldb, sB, n, nrhs, true, o.layout))
        return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    GLASS_TRY(placement_of(GLASS_OP_TRSM, n, nrhs, batch, o, pl));
    return from_cuda(launch_trsm(n, nrhs, make_mat(L, lda, sA, n, n, o.layout),
                                 make_mat(B, ldb, sB, n, nrhs, o.layout), batch, pl,
                                 reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_getrf_getrs(int n, int nrhs, void *A, int lda, long long sA, int *ipiv, void *B, int ldb,
                                       long long sB, int *info, int batch, const glass_opts *opts,
                                       glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    GLASS_TRY(check_order(n));
    if (nrhs < 0 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (batch == 0) return GLASS_OK;
    if (o.dtype == GLASS_F64) {
        if (!operand_ok(A, lda, sA, n, n, true, o.layout) || ipiv == nullptr || info == nullptr)
            return GLASS_ERR_INVALID_VALUE;
        if (nrhs > 0 && !operand_ok(B, ldb, sB, n, nrhs, true, o.layout)) return GLASS_ERR_INVALID_VALUE;
        Placement pl;
        GLASS_TRY(f64_placement_of(GLASS_OP_GETRF_GETRS, n, batch, o, pl));
        return from_cuda(launch_lu_f64(n, nrhs, static_cast<double *>(A), lda, sA, ipiv, static_cast<double *>(B),
                                       ldb, sB, info, batch, pl, reinterpret_cast<cudaStream_t>(stream)));
    }
    if (o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!operand_ok(A, lda, sA, n, n, true, o.layout) || ipiv == nullptr || info == nullptr)
        return GLASS_ERR_INVALID_VALUE;
    if (nrhs > 0 && !operand_ok(B, ldb, sB, n, nrhs, true, o.layout)) return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    GLASS_TRY(placement_of(GLASS_OP_GETRF_GETRS, n, nrhs, batch, o, pl));
    const Mat Bm = nrhs > 0 ? make_mat(B, ldb, sB, n, nrhs, o.layout) : make_mat(A, lda, sA, n, n, o.layout);
    return from_cuda(launch_getrf_getrs(n, nrhs, make_mat(A, lda, sA, n, n, o.layout), ipiv, Bm, info, batch, pl,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_rot3_compose(int chain, const void *Rs, long long sRs, void *R, long long sR, int batch,
                                        const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (chain < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (chain > 64) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.layout != GLASS_LAYOUT_COLMAJOR || o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!Rs || !R || sRs < 0 || sR < 9) return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    GLASS_TRY(placement_of(GLASS_OP_ROT3, 3, chain, batch, o, pl));
    return from_cuda(launch_rot3(chain, make_mat(Rs, 3, sRs, 3, 3 * chain, GLASS_LAYOUT_COLMAJOR),
                                 make_mat(R, 3, sR, 3, 3, GLASS_LAYOUT_COLMAJOR), batch, pl,
                                 reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_se3_apply(int chain, const void *T, long long sT, int npts, const void *P, long long sP,
                                     void *Q, long long sQ, int batch, const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (chain < 1 || npts < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (chain > 64) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.layout != GLASS_LAYOUT_COLMAJOR || o.dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (!T || !P || !Q || sT < 0 || sP < 0 || sQ < 3LL * npts) return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    GLASS_TRY(placement_of(GLASS_OP_SE3, 4, chain, batch, o, pl));
    return from_cuda(launch_se3(chain, make_mat(T, 4, sT, 4, 4 * chain, GLASS_LAYOUT_COLMAJOR), npts,
                                make_mat(P, 3, sP, 3, npts, GLASS_LAYOUT_COLMAJOR),
                                make_mat(Q, 3, sQ, 3, npts, GLASS_LAYOUT_COLMAJOR), batch, pl,
                                reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_to_interleaved32(int rows, int cols, const float *src, float *dst, int batch,
                                    glass_stream_t stream) {
    if (rows < 1 || cols < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if ((long long)rows * cols > (1 << 24)) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (!src || !dst) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_to_interleaved(rows, cols, src, dst, batch, reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_from_interleaved32(int rows, int cols, const float *src, float *dst, int batch,
                                      glass_stream_t stream) {
    if (rows < 1 || cols < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if ((long long)rows * cols > (1 << 24)) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (!src || !dst) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_from_interleaved(rows, cols, src, dst, batch, reinterpret_cast<cudaStream_t>(stream)));
}

size_t glass_posv_varsize_workspace(int batch) { return batch <= 0 ? 256 : varsize_workspace(batch); }

glass_status glass_posv_varsize(int batch, const int *n_dev, const long long *offA_dev, const long long *offB_dev,
                                int nrhs, void *A, void *B, int *info, void *ws, size_t ws_bytes,
                                const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (batch < 0 || nrhs < 1) return GLASS_ERR_INVALID_VALUE;
    if (nrhs > 16) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.layout != GLASS_LAYOUT_COLMAJOR) return GLASS_ERR_UNSUPPORTED;
    if (!n_dev || !offA_dev || !offB_dev || !A || !B || !info) return GLASS_ERR_INVALID_VALUE;
    if (!ws || ws_bytes < varsize_workspace(batch) || (reinterpret_cast<uintptr_t>(ws) & 255))
        return GLASS_ERR_WORKSPACE;
    int wpc = 8;
    if (o.placement.scope == GLASS_SCOPE_WARP && o.placement.pack != 0) {
        if (!valid_pack(o.placement.pack)) return GLASS_ERR_INVALID_VALUE;
        wpc = o.placement.pack;
    } else if (o.placement.scope != GLASS_SCOPE_AUTO) {
        return GLASS_ERR_UNSUPPORTED;
    }
    unsigned *status = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void **>(&status), g_device_status) != cudaSuccess)
        return GLASS_ERR_CUDA;
    return from_cuda(launch_posv_varsize(batch, n_dev, offA_dev, offB_dev, nrhs, static_cast<float *>(A),
                                         static_cast<float *>(B), info, ws, wpc, status,
                                         reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_gemm_ex(int transa, int transb, int m, int n, int k, float alpha, const void *A, int lda,
                                   long long sA, const void *B, int ldb, long long sB, float beta, void *C, int ldc,
                                   long long sC, int batch, const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if ((transa != 0 && transa != 1) || (transb != 0 && transb != 1) || m < 1 || n < 1 || k < 1 || batch < 0)
        return GLASS_ERR_INVALID_VALUE;
    if (m > 64 || n > 64 || k > 64) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    const int ra = transa ? k : m, ca = transa ? m : k, rb = transb ? n : k, cb = transb ? k : n;
    if (!operand_ok(A, lda, sA, ra, ca, false, o.layout) || !operand_ok(B, ldb, sB, rb, cb, false, o.layout) ||
        !operand_ok(C, ldc, sC, m, n, true, o.layout))
        return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    if (o.placement.scope == GLASS_SCOPE_AUTO) {
        pl = m * n <= 512 ? Placement{SCOPE_WARP, 4} : Placement{SCOPE_BLOCK, 1};
        if (o.placement.pack != 0) {
            if (!valid_pack(o.placement.pack)) return GLASS_ERR_INVALID_VALUE;
            pl.pack = o.placement.pack;
        }
        while (!feasible_gemm_ex(transa, transb, m, n, k, pl) && pl.pack > 1) pl.pack >>= 1;
    } else {
        if (o.placement.scope != GLASS_SCOPE_WARP && o.placement.scope != GLASS_SCOPE_BLOCK)
            return GLASS_ERR_INVALID_VALUE;
        pl = Placement{o.placement.scope, o.placement.pack == 0 ? 1 : o.placement.pack};
        if (!valid_pack(pl.pack)) return GLASS_ERR_INVALID_VALUE;
    }
    if (!feasible_gemm_ex(transa, transb, m, n, k, pl)) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_gemm_ex(transa, transb, m, n, k, alpha, make_mat(A, lda, sA, ra, ca, o.layout),
                                    make_mat(B, ldb, sB, rb, cb, o.layout), beta, make_mat(C, ldc, sC, m, n, o.layout),
                                    batch, pl, reinterpret_cast<cudaStream_t>(stream)));
}

size_t glass_riccati_workspace(int nx, int nu, int batch) {
    if (nx < 1 || nu < 1 || nx > 64 || nu > 64 || batch < 0) return 0;
    return ric_workspace(nx, nu, batch);
}

glass_status glass_riccati_gain(int nx, int nu, const void *A, long long sA, const void *B, long long sB, const void *P,
                                long long sP, const void *R, long long sR, void *K, long long sK, int *info, int batch,
                                void *ws, size_t ws_bytes, const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (nx < 1 || nu < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (nx > 64 || nu > 64) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    if (!A || !B || !P || !R || !K || !info) return GLASS_ERR_INVALID_VALUE;
    if (sA < 0 || sB < 0 || sP < 0 || sR < 0 || sK < (long long)nu * nx) return GLASS_ERR_INVALID_VALUE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the composition copies each problem's R: it needs sR >= nu * nu
    const bool ws_ok = ws != nullptr && ws_bytes >= ric_workspace(nx, nu, batch) &&
                       (reinterpret_cast<uintptr_t>(ws) & 255) == 0 && sR >= (long long)nu * nu;
    Placement pl;
    if (o.placement.scope == GLASS_SCOPE_AUTO) {
        pl = ric_resolve(nx, nu, batch, ws_ok);
        if (o.placement.pack != 0 && pl.scope != GLASS_SCOPE_COMPOSED) {
            if (!valid_pack(o.placement.pack)) return GLASS_ERR_INVALID_VALUE;
            pl.pack = o.placement.pack;
        }
    } else if (o.placement.scope == GLASS_SCOPE_COMPOSED) {
        if (!ws_ok) return GLASS_ERR_WORKSPACE;
        pl = Placement{GLASS_SCOPE_COMPOSED, 1};
    } else {
        if (o.placement.scope != GLASS_SCOPE_WARP && o.placement.scope != GLASS_SCOPE_BLOCK)
            return GLASS_ERR_INVALID_VALUE;
        pl = Placement{o.placement.scope, o.placement.pack == 0 ? 1 : o.placement.pack};
        if (!valid_pack(pl.pack)) return GLASS_ERR_INVALID_VALUE;
    }
    if (pl.scope == GLASS_SCOPE_COMPOSED) {
        // one call per primitive, each with its own measured placement
        float *PB = static_cast<float *>(ws);
        float *S = PB + ((size_t)batch * nx * nu + 63) / 64 * 64;
        const glass_opts a = kDefaultOpts;
        const long long sPB = (long long)nx * nu, sS = (long long)nu * nu;
        GLASS_TRY(glass_batched_gemm(nx, nu, nx, P, nx, sP, B, nx, sB, PB, nx, sPB, batch, &a, stream));
        if (cudaMemcpy2DAsync(S, (size_t)sS * 4, R, (size_t)sR * 4, (size_t)sS * 4, (size_t)batch,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return GLASS_ERR_CUDA;
        GLASS_TRY(glass_batched_gemm_ex(1, 0, nu, nu, nx, 1.f, B, nx, sB, PB, nx, sPB, 1.f, S, nu, sS, batch, &a,
                                        stream));
        GLASS_TRY(glass_batched_gemm_ex(1, 0, nu, nx, nx, 1.f, PB, nx, sPB, A, nx, sA, 0.f, K, nu, sK, batch, &a,
                                        stream));
        return glass_batched_posv(nu, nx, S, nu, sS, K, nu, sK, info, batch, &a, stream);
    }
    if (!feasible_riccati(nx, nu, pl)) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_riccati(nx, nu, static_cast<const float *>(A), sA, static_cast<const float *>(B), sB,
                                    static_cast<const float *>(P), sP, static_cast<const float *>(R), sR,
                                    static_cast<float *>(K), sK, info, batch, pl, st));
}

glass_status glass_riccati_placement(int nx, int nu, int batch, int composed_ok, glass_placement *out) {
    if (out == nullptr || nx < 1 || nu < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (nx > 64 || nu > 64) return GLASS_ERR_UNSUPPORTED;
    const Placement pl = ric_resolve(nx, nu, batch, composed_ok != 0);
    out->scope = pl.scope;
    out->pack = pl.pack;
    return GLASS_OK;
}

int glass_riccati_feasible(int nx, int nu, glass_placement p) {
    return feasible_riccati(nx, nu, Placement{p.scope, p.pack}) ? 1 : 0;
}

#define GLASS_ROBO_ENTRY(op, n, a, b, sa, o1, o2, o3, so, idx)                                           \
    const glass_opts &o = opts_or_default(opts);                                                          \
    GLASS_TRY(check_common(o));                                                                           \
    if (batch < 0) return GLASS_ERR_INVALID_VALUE;                                                        \
    if (batch == 0) return GLASS_OK;                                                                      \
    Placement pl;                                                                                         \
    GLASS_TRY(robo_placement_of(op, n, batch, o, pl));                                                    \
    return from_cuda(launch_robo(op, n, static_cast<const float *>(a), static_cast<const float *>(b), sa,  \
                                 static_cast<float *>(o1), static_cast<float *>(o2), static_cast<float *>(o3), \
                                 so, idx, batch, pl, reinterpret_cast<cudaStream_t>(stream)))

glass_status glass_batched_quat_retract(const void *q, const void *d, void *out, int batch, const glass_opts *opts,
                                        glass_stream_t stream) {
    if (batch > 0 && (!q || !d || !out || !aligned16(q) || !aligned16(out))) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_QUAT_RETRACT, 0, q, d, 0, out, nullptr, nullptr, 0, nullptr);
}

glass_status glass_batched_quat_error(const void *q1, const void *q2, void *out, int batch, const glass_opts *opts,
                                      glass_stream_t stream) {
    if (batch > 0 && (!q1 || !q2 || !out || !aligned16(q1) || !aligned16(q2))) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_QUAT_ERROR, 0, q1, q2, 0, out, nullptr, nullptr, 0, nullptr);
}

glass_status glass_batched_se3_retract(const void *T, const void *xi, void *out, int batch, const glass_opts *opts,
                                       glass_stream_t stream) {
    if (batch > 0 && (!T || !xi || !out || !aligned16(T) || !aligned16(out))) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_SE3_RETRACT, 0, T, xi, 0, out, nullptr, nullptr, 0, nullptr);
}

glass_status glass_batched_motion_cross(const void *v, const void *m, void *out, int batch, const glass_opts *opts,
                                        glass_stream_t stream) {
    if (batch > 0 && (!v || !m || !out)) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_MOTION_CROSS, 0, v, m, 0, out, nullptr, nullptr, 0, nullptr);
}

glass_status glass_batched_eig3(const void *A, void *w, void *V, int batch, const glass_opts *opts,
                                glass_stream_t stream) {
    if (batch > 0 && (!A || !w || !V)) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_EIG3, 0, A, nullptr, 0, w, V, nullptr, 0, nullptr);
}

glass_status glass_batched_svd3(const void *M, void *U, void *sv, void *V, int batch, const glass_opts *opts,
                                glass_stream_t stream) {
    if (batch > 0 && (!M || !U || !sv || !V)) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_SVD3, 0, M, nullptr, 0, U, sv, V, 0, nullptr);
}

glass_status glass_batched_closest_rotation(const void *M, void *R, int batch, const glass_opts *opts,
                                            glass_stream_t stream) {
    if (batch > 0 && (!M || !R)) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_CLOSEST_ROTATION, 0, M, nullptr, 0, R, nullptr, nullptr, 0, nullptr);
}

glass_status glass_batched_argmax(int n, const void *x, long long sx, int *idx, int batch, const glass_opts *opts,
                                  glass_stream_t stream) {
    if (n < 1 || (batch > 0 && (!x || !idx || sx < 0 || (batch > 1 && sx < n)))) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_ARGMAX, n, x, nullptr, sx, nullptr, nullptr, nullptr, 0, idx);
}

glass_status glass_batched_softmax(int n, const void *x, long long sx, void *y, long long sy, int batch,
                                   const glass_opts *opts, glass_stream_t stream) {
    if (n < 1 || (batch > 0 && (!x || !y || sx < 0 || sy < n))) return GLASS_ERR_INVALID_VALUE;
    GLASS_ROBO_ENTRY(ROBO_SOFTMAX, n, x, nullptr, sx, y, nullptr, nullptr, sy, nullptr);
}
#undef GLASS_ROBO_ENTRY

glass_status glass_batched_dot(int n, const void *x, long long sx, const void *y, long long sy, void *out, int batch,
                               const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (n < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    if (!x || !y || !out || sx < 0 || sy < 0) return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    if (o.placement.scope == GLASS_SCOPE_AUTO) {
        pl = n <= 32 ? Placement{SCOPE_THREAD, 4} : n <= 512 ? Placement{SCOPE_WARP, 4} : Placement{SCOPE_BLOCK, 2};
        if (o.placement.pack != 0) pl.pack = o.placement.pack;
    } else {
        pl = Placement{o.placement.scope, o.placement.pack == 0 ? 1 : o.placement.pack};
    }
    if (pl.scope < SCOPE_THREAD || pl.scope > SCOPE_BLOCK || !valid_pack(pl.pack) ||
        (pl.scope == SCOPE_BLOCK && pl.pack > 4))
        return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_dot(n, static_cast<const float *>(x), sx, static_cast<const float *>(y), sy,
                                static_cast<float *>(out), batch, pl, reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_gemv(int trans, int m, int n, float alpha, const void *A, int lda, long long sA,
                                const void *x, long long sx, float beta, void *y, long long sy, int batch,
                                const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if ((trans != 0 && trans != 1) || m < 1 || n < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (m > 64 || n > 64) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    const int ylen = trans ? n : m;
    if (!operand_ok(A, lda, sA, m, n, false, o.layout) || !x || !y || sx < 0 || sy < ylen)
        return GLASS_ERR_INVALID_VALUE;
    Placement pl;
    if (o.placement.scope == GLASS_SCOPE_AUTO) {
        pl = m * n <= 64 ? Placement{SCOPE_THREAD, 2} : Placement{SCOPE_WARP, 4};
        if (o.placement.pack != 0) pl.pack = o.placement.pack;
    } else {
        pl = Placement{o.placement.scope, o.placement.pack == 0 ? 1 : o.placement.pack};
    }
    if ((pl.scope != SCOPE_THREAD && pl.scope != SCOPE_WARP) || !valid_pack(pl.pack)) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_gemv(trans, m, n, alpha, make_mat(A, lda, sA, m, n, o.layout),
                                 static_cast<const float *>(x), sx, beta, static_cast<float *>(y), sy, batch, pl,
                                 reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_trsv(int n, const void *L, int lda, long long sA, void *x, long long sx, int batch,
                                const glass_opts *opts, glass_stream_t stream) {
    return glass_batched_trsm(n, 1, L, lda, sA, x, n, sx, batch, opts, stream);
}

glass_status glass_batched_btd_matvec(int nb, int N, const void *D, const void *O, const void *x, void *y, int batch,
                                      const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (nb < 1 || N < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (nb > 32) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    if (!D || (N > 1 && !O) || !x || !y) return GLASS_ERR_INVALID_VALUE;
    if (o.placement.scope != GLASS_SCOPE_AUTO && o.placement.scope != GLASS_SCOPE_WARP) return GLASS_ERR_INVALID_VALUE;
    const int pack = o.placement.pack == 0 ? 4 : o.placement.pack;
    if (!valid_pack(pack)) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_btd_matvec(nb, N, static_cast<const float *>(D), static_cast<const float *>(O),
                                       static_cast<const float *>(x), static_cast<float *>(y), batch, pack,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_batched_btd_posv(int nb, int N, void *D, void *O, void *b, int *info, int batch,
                                    const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (nb < 1 || N < 1 || batch < 0) return GLASS_ERR_INVALID_VALUE;
    if (nb > 32) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    if (!D || (N > 1 && !O) || !b || !info) return GLASS_ERR_INVALID_VALUE;
    if (o.placement.scope != GLASS_SCOPE_AUTO && o.placement.scope != GLASS_SCOPE_WARP) return GLASS_ERR_INVALID_VALUE;
    const int pack = o.placement.pack == 0 ? 2 : o.placement.pack;
    if (!valid_pack(pack)) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_btd_posv(nb, N, static_cast<float *>(D), static_cast<float *>(O), static_cast<float *>(b),
                                     info, batch, pack, reinterpret_cast<cudaStream_t>(stream)));
}

size_t glass_btd_pcg_workspace(int nb, int N, int batch) {
    if (nb < 1 || N < 1 || batch < 0) return 0;
    return (size_t)batch * N * nb * nb * sizeof(float);
}

glass_status glass_batched_btd_pcg(int nb, int N, const void *D, const void *O, const void *b, void *x, int iters,
                                   float tol, int *iters_done, void *ws, size_t ws_bytes, int batch,
                                   const glass_opts *opts, glass_stream_t stream) {
    const glass_opts &o = opts_or_default(opts);
    GLASS_TRY(check_common(o));
    if (nb < 1 || N < 1 || batch < 0 || iters < 0 || !(tol >= 0.f)) return GLASS_ERR_INVALID_VALUE;
    if (nb > 32 || N > 64) return GLASS_ERR_UNSUPPORTED;
    if (batch == 0) return GLASS_OK;
    if (o.dtype != GLASS_F32 || o.math != GLASS_MATH_FP32 || o.layout != GLASS_LAYOUT_COLMAJOR)
        return GLASS_ERR_UNSUPPORTED;
    if (!D || (N > 1 && !O) || !b || !x || !iters_done) return GLASS_ERR_INVALID_VALUE;
    if (!ws || ws_bytes < glass_btd_pcg_workspace(nb, N, batch) || (reinterpret_cast<uintptr_t>(ws) & 15) != 0)
        return GLASS_ERR_WORKSPACE;
    if (o.placement.scope != GLASS_SCOPE_AUTO && o.placement.scope != GLASS_SCOPE_WARP) return GLASS_ERR_INVALID_VALUE;
    int pack = o.placement.pack;
    if (pack == 0) {  // as many warps per CTA (up to 4) as fit the per-CTA shared memory
        pack = 4;
        while (pack > 1 && btd_pcg_smem(nb, N, pack) > 100 * 1024) pack >>= 1;
    }
    if (!valid_pack(pack)) return GLASS_ERR_INVALID_VALUE;
    if (btd_pcg_smem(nb, N, pack) > 227 * 1024) return GLASS_ERR_UNSUPPORTED;
    return from_cuda(launch_btd_pcg(nb, N, static_cast<const float *>(D), static_cast<const float *>(O),
                                    static_cast<const float *>(b), static_cast<float *>(x), iters, tol, iters_done,
                                    static_cast<float *>(ws), batch, pack, reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_robo_placement(int op, int n, int batch, glass_placement *out) {
    if (out == nullptr || op < 0 || op >= GLASS_ROBO_NUM_OPS || batch < 0) return GLASS_ERR_INVALID_VALUE;
    const Placement pl = robo_resolve(op, n < 1 ? 1 : n, batch);
    out->scope = pl.scope;
    out->pack = pl.pack;
    return GLASS_OK;
}

int glass_robo_feasible(int op, int n, glass_placement p) {
    if (op < 0 || op >= GLASS_ROBO_NUM_OPS) return 0;
    return feasible_robo(op, n, Placement{p.scope, p.pack}) ? 1 : 0;
}

glass_status glass_get_placement(int op, int n, int k, int batch, int dtype, int use_learned, glass_placement *out) {
    if (out == nullptr || op < 0 || op >= GLASS_NUM_OPS || batch < 0 || k < 0) return GLASS_ERR_INVALID_VALUE;
    if (dtype != GLASS_F32) return GLASS_ERR_UNSUPPORTED;
    if (op == GLASS_OP_ROT3 || op == GLASS_OP_SE3) {
        if (k < 1 || k > 64) return GLASS_ERR_INVALID_VALUE;
    } else {
        GLASS_TRY(check_order(n));
    }
    const Placement pl = resolve(op, n, k > 0 ? k : 1, batch, use_learned);
    out->scope = pl.scope;
    out->pack = pl.pack;
    return GLASS_OK;
}

int glass_placement_feasible(int op, int n, int k, glass_placement p) {
    if (op < 0 || op >= GLASS_NUM_OPS) return 0;
    return feasible(op, n, k, Placement{p.scope, p.pack}) ? 1 : 0;
}

glass_status glass_set_learned_model(const float *weights, int nweights, const float *feat_mean,
                                     const float *feat_std) {
    if (!weights || nweights != 5516 || !feat_mean || !feat_std) return GLASS_ERR_INVALID_VALUE;
    for (int i = 0; i < 8; ++i)
        if (!(feat_std[i] > 0.f)) return GLASS_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lk(g_learned_mu);
    memcpy(g_learned.w, weights, sizeof(g_learned.w));
    memcpy(g_learned.mean, feat_mean, sizeof(g_learned.mean));
    memcpy(g_learned.stdv, feat_std, sizeof(g_learned.stdv));
    g_learned.set = true;
    return GLASS_OK;
}

size_t glass_mlp_workspace(int rows) { return rows <= 0 ? 256 : mlp_workspace(rows); }

glass_status glass_mlp_forward(int din, const float *w, int rows, const float *X, float *Y, glass_stream_t stream) {
    if (din != 8 || rows < 0) return din != 8 ? GLASS_ERR_UNSUPPORTED : GLASS_ERR_INVALID_VALUE;
    if (rows == 0) return GLASS_OK;
    if (!w || !X || !Y) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_mlp_forward(din, w, rows, X, Y, reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_mlp_loss_grad(int din, const float *w, int rows, const float *X, const float *T, const float *M,
                                 float *grad, float *loss_dev, void *ws, size_t ws_bytes, glass_stream_t stream) {
    if (din != 8) return GLASS_ERR_UNSUPPORTED;
    if (rows < 1 || !w || !X || !T || !M || !grad || !loss_dev) return GLASS_ERR_INVALID_VALUE;
    if (!ws || ws_bytes < mlp_workspace(rows) || (reinterpret_cast<uintptr_t>(ws) & 255)) return GLASS_ERR_WORKSPACE;
    return from_cuda(launch_mlp_loss_grad(din, w, rows, X, T, M, grad, loss_dev, ws,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_mlp_adam(int nparams, float *w, const float *grad, float *m, float *v, int t, float lr, float beta1,
                            float beta2, float eps, glass_stream_t stream) {
    if (nparams < 0 || t < 1 || !(lr > 0.f) || !(eps > 0.f)) return GLASS_ERR_INVALID_VALUE;
    if (nparams == 0) return GLASS_OK;
    if (!w || !grad || !m || !v) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_mlp_adam(nparams, w, grad, m, v, t, lr, beta1, beta2, eps,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

glass_status glass_last_device_status(glass_stream_t stream) {
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return GLASS_ERR_CUDA;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_device_status, sizeof v) != cudaSuccess) return GLASS_ERR_CUDA;
    const unsigned zero = 0;
    if (cudaMemcpyToSymbol(g_device_status, &zero, sizeof zero) != cudaSuccess) return GLASS_ERR_CUDA;
    return v == 0 ? GLASS_OK : (glass_status)v;
}

glass_status glass_selftest_wait_timeout(const float *A, const float *B, float *C, int batch, long long wait_cycles,
                                         glass_stream_t stream) {
    if (batch < 0 || wait_cycles < 1 || wait_cycles > (1ll << 31)) return GLASS_ERR_INVALID_VALUE;
    if (batch == 0) return GLASS_OK;
    if (!A || !B || !C) return GLASS_ERR_INVALID_VALUE;
    return from_cuda(launch_gemm_umma64_ex(A, B, C, batch, wait_cycles, 1, reinterpret_cast<cudaStream_t>(stream)));
}

const char *glass_status_string(glass_status s) {
    switch (s) {
        case GLASS_OK: return "GLASS_OK";
        case GLASS_ERR_INVALID_VALUE: return "GLASS_ERR_INVALID_VALUE";
        case GLASS_ERR_UNSUPPORTED: return "GLASS_ERR_UNSUPPORTED";
        case GLASS_ERR_CUDA: return "GLASS_ERR_CUDA";
        case GLASS_ERR_TIMEOUT: return "GLASS_ERR_TIMEOUT";
        case GLASS_ERR_WORKSPACE: return "GLASS_ERR_WORKSPACE";
        default: return "GLASS_ERR_UNKNOWN";
    }
}

const char *glass_version(void) { return "glass sm_103a"; }

}  // extern "C"
