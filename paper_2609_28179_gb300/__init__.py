"""GB300-native (sm_103a) batched small-matrix linear algebra: the GLASS hot
path (arxiv 2609.28179) behind a C ABI.

This module is a thin ctypes binding of ``libglass.so`` (see include/glass.h
for every contract).  Each ``glass_*`` function has the C name, takes the C
arguments in the C order, and returns the integer ``glass_status``; tensors
may be passed wherever the C function takes a device pointer (their
``data_ptr()`` is used), and ``stream=None`` means torch's current stream.
Every computation runs in the library's CUDA kernels: there is no host or
PyTorch fallback, and loading fails loudly when the library is not built.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglass.so")

# status codes
GLASS_OK = 0
GLASS_ERR_INVALID_VALUE = 1
GLASS_ERR_UNSUPPORTED = 2
GLASS_ERR_CUDA = 3
GLASS_ERR_TIMEOUT = 4
GLASS_ERR_WORKSPACE = 5
# dtypes / math / layouts / scopes / ops
GLASS_F32, GLASS_F64, GLASS_BF16 = 0, 1, 2
GLASS_MATH_FP32, GLASS_MATH_BF16_TC, GLASS_MATH_TF32_TC, GLASS_MATH_3XTF32_TC = 0, 1, 2, 3
GLASS_LAYOUT_COLMAJOR, GLASS_LAYOUT_INTERLEAVED32 = 0, 1
GLASS_RESIDUAL_FP64, GLASS_RESIDUAL_DOT2 = 0, 1
GLASS_SCOPE_AUTO, GLASS_SCOPE_THREAD, GLASS_SCOPE_WARP, GLASS_SCOPE_BLOCK, GLASS_SCOPE_COMPOSED = -1, 0, 1, 2, 3
(GLASS_OP_GEMM, GLASS_OP_POSV, GLASS_OP_TRSM, GLASS_OP_GETRF_GETRS, GLASS_OP_ROT3, GLASS_OP_SE3,
 GLASS_OP_POTRF, GLASS_OP_POTRS) = range(8)
SCOPE_NAMES = {0: "thread", 1: "warp", 2: "block", 3: "composed"}
# robotics operations (glass_robo_op)
ROBO_OPS = ["quat_retract", "quat_error", "se3_retract", "motion_cross", "eig3", "svd3", "closest_rotation",
            "argmax", "softmax"]
# The 12 placements of the table / cost model, index = scope*4 + log2(pack).
PLACEMENTS = [(s, p) for s in (0, 1, 2) for p in (1, 2, 4, 8)]


class GlassError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class glass_placement(ctypes.Structure):
    _fields_ = [("scope", ctypes.c_int), ("pack", ctypes.c_int)]


class glass_opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("math", ctypes.c_int), ("layout", ctypes.c_int),
                ("placement", glass_placement), ("refine_steps", ctypes.c_int),
                ("fp64_diag", ctypes.c_int), ("use_learned", ctypes.c_int), ("residual", ctypes.c_int)]


def make_opts(dtype=GLASS_F32, math=GLASS_MATH_FP32, layout=GLASS_LAYOUT_COLMAJOR, scope=GLASS_SCOPE_AUTO,
              pack=0, refine_steps=0, fp64_diag=0, use_learned=0, residual=GLASS_RESIDUAL_FP64) -> glass_opts:
    return glass_opts(dtype, math, layout, glass_placement(scope, pack), refine_steps, fp64_diag, use_learned,
                      residual)


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_i = ctypes.c_int
_ll = ctypes.c_longlong
_sz = ctypes.c_size_t
_f = ctypes.c_float
_OPTS = ctypes.POINTER(glass_opts)
_SIGS = {
    "glass_batched_gemm": (_i, [_i, _i, _i, _P, _i, _ll, _P, _i, _ll, _P, _i, _ll, _i, _OPTS, _P]),
    "glass_batched_potrf": (_i, [_i, _P, _i, _ll, _P, _i, _OPTS, _P]),
    "glass_batched_potrs": (_i, [_i, _i, _P, _i, _ll, _P, _i, _ll, _i, _OPTS, _P]),
    "glass_batched_posv": (_i, [_i, _i, _P, _i, _ll, _P, _i, _ll, _P, _i, _OPTS, _P]),
    "glass_batched_trsm": (_i, [_i, _i, _P, _i, _ll, _P, _i, _ll, _i, _OPTS, _P]),
    "glass_batched_getrf_getrs": (_i, [_i, _i, _P, _i, _ll, _P, _P, _i, _ll, _P, _i, _OPTS, _P]),
    "glass_batched_rot3_compose": (_i, [_i, _P, _ll, _P, _ll, _i, _OPTS, _P]),
    "glass_batched_se3_apply": (_i, [_i, _P, _ll, _i, _P, _ll, _P, _ll, _i, _OPTS, _P]),
    "glass_to_interleaved32": (_i, [_i, _i, _P, _P, _i, _P]),
    "glass_from_interleaved32": (_i, [_i, _i, _P, _P, _i, _P]),
    "glass_posv_varsize_workspace": (_sz, [_i]),
    "glass_posv_varsize": (_i, [_i, _P, _P, _P, _i, _P, _P, _P, _P, _sz, _OPTS, _P]),
    "glass_posv_varsize_noalloc": (_i, [_i, _P, _P, _P, _i, _P, _P, _P, _OPTS, _P]),
    "glass_get_placement": (_i, [_i, _i, _i, _i, _i, _i, ctypes.POINTER(glass_placement)]),
    "glass_placement_feasible": (_i, [_i, _i, _i, glass_placement]),
    "glass_set_learned_model": (_i, [_P, _i, _P, _P]),
    "glass_mlp_workspace": (_sz, [_i]),
    "glass_mlp_forward": (_i, [_i, _P, _i, _P, _P, _P]),
    "glass_mlp_loss_grad": (_i, [_i, _P, _i, _P, _P, _P, _P, _P, _P, _sz, _P]),
    "glass_mlp_adam": (_i, [_i, _P, _P, _P, _P, _i, _f, _f, _f, _f, _P]),
    "glass_last_device_status": (_i, [_P]),
    "glass_selftest_wait_timeout": (_i, [_P, _P, _P, _i, _ll, _P]),
    "glass_batched_gemm_ex": (_i, [_i, _i, _i, _i, _i, ctypes.c_float, _P, _i, _ll, _P, _i, _ll, ctypes.c_float,
                                   _P, _i, _ll, _i, _OPTS, _P]),
    "glass_riccati_workspace": (ctypes.c_size_t, [_i, _i, _i]),
    "glass_riccati_gain": (_i, [_i, _i, _P, _ll, _P, _ll, _P, _ll, _P, _ll, _P, _ll, _P, _i, _P, ctypes.c_size_t,
                                _OPTS, _P]),
    "glass_riccati_placement": (_i, [_i, _i, _i, _i, ctypes.POINTER(glass_placement)]),
    "glass_riccati_feasible": (_i, [_i, _i, glass_placement]),
    "glass_batched_quat_retract": (_i, [_P, _P, _P, _i, _OPTS, _P]),
    "glass_batched_quat_error": (_i, [_P, _P, _P, _i, _OPTS, _P]),
    "glass_batched_se3_retract": (_i, [_P, _P, _P, _i, _OPTS, _P]),
    "glass_batched_motion_cross": (_i, [_P, _P, _P, _i, _OPTS, _P]),
    "glass_batched_eig3": (_i, [_P, _P, _P, _i, _OPTS, _P]),
    "glass_batched_svd3": (_i, [_P, _P, _P, _P, _i, _OPTS, _P]),
    "glass_batched_closest_rotation": (_i, [_P, _P, _i, _OPTS, _P]),
    "glass_batched_argmax": (_i, [_i, _P, _ll, _P, _i, _OPTS, _P]),
    "glass_batched_softmax": (_i, [_i, _P, _ll, _P, _ll, _i, _OPTS, _P]),
    "glass_batched_dot": (_i, [_i, _P, _ll, _P, _ll, _P, _i, _OPTS, _P]),
    "glass_batched_gemv": (_i, [_i, _i, _i, ctypes.c_float, _P, _i, _ll, _P, _ll, ctypes.c_float, _P, _ll, _i,
                                _OPTS, _P]),
    "glass_batched_trsv": (_i, [_i, _P, _i, _ll, _P, _ll, _i, _OPTS, _P]),
    "glass_batched_btd_matvec": (_i, [_i, _i, _P, _P, _P, _P, _i, _OPTS, _P]),
    "glass_batched_btd_posv": (_i, [_i, _i, _P, _P, _P, _P, _i, _OPTS, _P]),
    "glass_btd_pcg_workspace": (_sz, [_i, _i, _i]),
    "glass_batched_btd_pcg": (_i, [_i, _i, _P, _P, _P, _P, _i, _f, _P, _P, _sz, _i, _OPTS, _P]),
    "glass_robo_placement": (_i, [_i, _i, _i, ctypes.POINTER(glass_placement)]),
    "glass_robo_feasible": (_i, [_i, _i, glass_placement]),
    "glass_peak_probe": (_i, [_i, _i, _i, _i, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "glass_status_string": (ctypes.c_char_p, [_i]),
    "glass_version": (ctypes.c_char_p, []),
}


def lib():
    """Load libglass.so (built by ``_build.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2609_28179_gb300._build.build() "
                               "(requires nvcc) -- there is no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def exported_symbols():
    return list(_SIGS)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, ctypes.c_void_p):
        return x.value
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _opts(o):
    return None if o is None else ctypes.byref(o)


def status_string(s: int) -> str:
    return lib().glass_status_string(int(s)).decode()


def check(status: int, what: str = "glass") -> None:
    if status != GLASS_OK:
        raise GlassError(status, what)


# ------------------------------------------------------------ entry points
def glass_batched_gemm(m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, batch, opts=None, stream=None):
    return lib().glass_batched_gemm(m, n, k, _ptr(A), lda, sA, _ptr(B), ldb, sB, _ptr(C), ldc, sC, batch,
                                    _opts(opts), _stream(stream))


def glass_batched_potrf(n, A, lda, sA, info, batch, opts=None, stream=None):
    return lib().glass_batched_potrf(n, _ptr(A), lda, sA, _ptr(info), batch, _opts(opts), _stream(stream))


def glass_batched_potrs(n, nrhs, L, lda, sA, B, ldb, sB, batch, opts=None, stream=None):
    return lib().glass_batched_potrs(n, nrhs, _ptr(L), lda, sA, _ptr(B), ldb, sB, batch, _opts(opts),
                                     _stream(stream))


def glass_batched_posv(n, nrhs, A, lda, sA, B, ldb, sB, info, batch, opts=None, stream=None):
    return lib().glass_batched_posv(n, nrhs, _ptr(A), lda, sA, _ptr(B), ldb, sB, _ptr(info), batch,
                                    _opts(opts), _stream(stream))


def glass_batched_trsm(n, nrhs, L, lda, sA, B, ldb, sB, batch, opts=None, stream=None):
    return lib().glass_batched_trsm(n, nrhs, _ptr(L), lda, sA, _ptr(B), ldb, sB, batch, _opts(opts),
                                    _stream(stream))


def glass_batched_getrf_getrs(n, nrhs, A, lda, sA, ipiv, B, ldb, sB, info, batch, opts=None, stream=None):
    return lib().glass_batched_getrf_getrs(n, nrhs, _ptr(A), lda, sA, _ptr(ipiv), _ptr(B), ldb, sB, _ptr(info),
                                           batch, _opts(opts), _stream(stream))


def glass_batched_rot3_compose(chain, Rs, sRs, R, sR, batch, opts=None, stream=None):
    return lib().glass_batched_rot3_compose(chain, _ptr(Rs), sRs, _ptr(R), sR, batch, _opts(opts),
                                            _stream(stream))


def glass_batched_se3_apply(chain, T, sT, npts, P, sP, Q, sQ, batch, opts=None, stream=None):
    return lib().glass_batched_se3_apply(chain, _ptr(T), sT, npts, _ptr(P), sP, _ptr(Q), sQ, batch,
                                         _opts(opts), _stream(stream))


def glass_to_interleaved32(rows, cols, src, dst, batch, stream=None):
    return lib().glass_to_interleaved32(rows, cols, _ptr(src), _ptr(dst), batch, _stream(stream))


def glass_from_interleaved32(rows, cols, src, dst, batch, stream=None):
    return lib().glass_from_interleaved32(rows, cols, _ptr(src), _ptr(dst), batch, _stream(stream))


def glass_posv_varsize_workspace(batch):
    return int(lib().glass_posv_varsize_workspace(batch))


def glass_posv_varsize(batch, n_dev, offA_dev, offB_dev, nrhs, A, B, info, ws, ws_bytes, opts=None,
                       stream=None):
    return lib().glass_posv_varsize(batch, _ptr(n_dev), _ptr(offA_dev), _ptr(offB_dev), nrhs, _ptr(A),
                                    _ptr(B), _ptr(info), _ptr(ws), ws_bytes, _opts(opts), _stream(stream))


def glass_posv_varsize_noalloc(batch, n_dev, offA_dev, offB_dev, nrhs, A, B, info, opts=None, stream=None):
    """Mixed-size solve with the library's built-in scratch (batch <= 65536),
    for callers that cannot allocate device memory."""
    return lib().glass_posv_varsize_noalloc(batch, _ptr(n_dev), _ptr(offA_dev), _ptr(offB_dev), nrhs, _ptr(A),
                                            _ptr(B), _ptr(info), _opts(opts), _stream(stream))


def glass_get_placement(op, n, k, batch, dtype=GLASS_F32, use_learned=0):
    """Returns (status, (scope, pack))."""
    out = glass_placement()
    s = lib().glass_get_placement(op, n, k, batch, dtype, use_learned, ctypes.byref(out))
    return s, (out.scope, out.pack)


def glass_placement_feasible(op, n, k, scope, pack):
    return bool(lib().glass_placement_feasible(op, n, k, glass_placement(scope, pack)))


def glass_set_learned_model(weights, feat_mean, feat_std):
    import numpy as np
    w = np.ascontiguousarray(weights, dtype=np.float32)
    mu = np.ascontiguousarray(feat_mean, dtype=np.float32)
    sd = np.ascontiguousarray(feat_std, dtype=np.float32)
    return lib().glass_set_learned_model(w.ctypes.data, w.size, mu.ctypes.data, sd.ctypes.data)


def glass_mlp_workspace(rows):
    return int(lib().glass_mlp_workspace(rows))


def glass_mlp_forward(din, w, rows, X, Y, stream=None):
    return lib().glass_mlp_forward(din, _ptr(w), rows, _ptr(X), _ptr(Y), _stream(stream))


def glass_mlp_loss_grad(din, w, rows, X, T, M, grad, loss_dev, ws, ws_bytes, stream=None):
    return lib().glass_mlp_loss_grad(din, _ptr(w), rows, _ptr(X), _ptr(T), _ptr(M), _ptr(grad),
                                     _ptr(loss_dev), _ptr(ws), ws_bytes, _stream(stream))


def glass_mlp_adam(nparams, w, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    return lib().glass_mlp_adam(nparams, _ptr(w), _ptr(grad), _ptr(m), _ptr(v), t, lr, beta1, beta2, eps,
                                _stream(stream))


def glass_last_device_status(stream=None):
    return lib().glass_last_device_status(_stream(stream))


def glass_selftest_wait_timeout(A, B, C, batch, wait_cycles, stream=None):
    return lib().glass_selftest_wait_timeout(_ptr(A), _ptr(B), _ptr(C), batch, wait_cycles, _stream(stream))


def glass_batched_gemm_ex(transa, transb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, opts=None,
                          stream=None):
    return lib().glass_batched_gemm_ex(transa, transb, m, n, k, alpha, _ptr(A), lda, sA, _ptr(B), ldb, sB, beta,
                                       _ptr(C), ldc, sC, batch, _opts(opts), _stream(stream))


def glass_riccati_workspace(nx, nu, batch):
    return lib().glass_riccati_workspace(nx, nu, batch)


def glass_riccati_gain(nx, nu, A, sA, B, sB, P, sP, R, sR, K, sK, info, batch, ws=None, ws_bytes=0, opts=None,
                       stream=None):
    return lib().glass_riccati_gain(nx, nu, _ptr(A), sA, _ptr(B), sB, _ptr(P), sP, _ptr(R), sR, _ptr(K), sK,
                                    _ptr(info), batch, _ptr(ws), ws_bytes, _opts(opts), _stream(stream))


def glass_riccati_placement(nx, nu, batch, composed_ok=True):
    """Returns (status, (scope, pack))."""
    out = glass_placement()
    s = lib().glass_riccati_placement(nx, nu, batch, int(bool(composed_ok)), ctypes.byref(out))
    return s, (out.scope, out.pack)


def glass_riccati_feasible(nx, nu, scope, pack):
    return bool(lib().glass_riccati_feasible(nx, nu, glass_placement(scope, pack)))


def glass_batched_quat_retract(q, d, out, batch, opts=None, stream=None):
    return lib().glass_batched_quat_retract(_ptr(q), _ptr(d), _ptr(out), batch, _opts(opts), _stream(stream))


def glass_batched_quat_error(q1, q2, out, batch, opts=None, stream=None):
    return lib().glass_batched_quat_error(_ptr(q1), _ptr(q2), _ptr(out), batch, _opts(opts), _stream(stream))


def glass_batched_se3_retract(T, xi, out, batch, opts=None, stream=None):
    return lib().glass_batched_se3_retract(_ptr(T), _ptr(xi), _ptr(out), batch, _opts(opts), _stream(stream))


def glass_batched_motion_cross(v, m, out, batch, opts=None, stream=None):
    return lib().glass_batched_motion_cross(_ptr(v), _ptr(m), _ptr(out), batch, _opts(opts), _stream(stream))


def glass_batched_eig3(A, w, V, batch, opts=None, stream=None):
    return lib().glass_batched_eig3(_ptr(A), _ptr(w), _ptr(V), batch, _opts(opts), _stream(stream))


def glass_batched_svd3(M, U, s, V, batch, opts=None, stream=None):
    return lib().glass_batched_svd3(_ptr(M), _ptr(U), _ptr(s), _ptr(V), batch, _opts(opts), _stream(stream))


def glass_batched_closest_rotation(M, R, batch, opts=None, stream=None):
    return lib().glass_batched_closest_rotation(_ptr(M), _ptr(R), batch, _opts(opts), _stream(stream))


def glass_batched_argmax(n, x, sx, idx, batch, opts=None, stream=None):
    return lib().glass_batched_argmax(n, _ptr(x), sx, _ptr(idx), batch, _opts(opts), _stream(stream))


def glass_batched_softmax(n, x, sx, y, sy, batch, opts=None, stream=None):
    return lib().glass_batched_softmax(n, _ptr(x), sx, _ptr(y), sy, batch, _opts(opts), _stream(stream))


def glass_batched_dot(n, x, sx, y, sy, out, batch, opts=None, stream=None):
    return lib().glass_batched_dot(n, _ptr(x), sx, _ptr(y), sy, _ptr(out), batch, _opts(opts), _stream(stream))


def glass_batched_gemv(trans, m, n, alpha, A, lda, sA, x, sx, beta, y, sy, batch, opts=None, stream=None):
    return lib().glass_batched_gemv(trans, m, n, alpha, _ptr(A), lda, sA, _ptr(x), sx, beta, _ptr(y), sy, batch,
                                    _opts(opts), _stream(stream))


def glass_batched_trsv(n, L, lda, sA, x, sx, batch, opts=None, stream=None):
    return lib().glass_batched_trsv(n, _ptr(L), lda, sA, _ptr(x), sx, batch, _opts(opts), _stream(stream))


def glass_batched_btd_matvec(nb, N, D, O, x, y, batch, opts=None, stream=None):
    return lib().glass_batched_btd_matvec(nb, N, _ptr(D), _ptr(O), _ptr(x), _ptr(y), batch, _opts(opts),
                                          _stream(stream))


def glass_batched_btd_posv(nb, N, D, O, b, info, batch, opts=None, stream=None):
    return lib().glass_batched_btd_posv(nb, N, _ptr(D), _ptr(O), _ptr(b), _ptr(info), batch, _opts(opts),
                                        _stream(stream))


def glass_btd_pcg_workspace(nb, N, batch):
    return lib().glass_btd_pcg_workspace(nb, N, batch)


def glass_batched_btd_pcg(nb, N, D, O, b, x, iters, tol, iters_done, ws, ws_bytes, batch, opts=None, stream=None):
    return lib().glass_batched_btd_pcg(nb, N, _ptr(D), _ptr(O), _ptr(b), _ptr(x), iters, tol, _ptr(iters_done),
                                       _ptr(ws), ws_bytes, batch, _opts(opts), _stream(stream))


def glass_robo_placement(op, n, batch):
    """Returns (status, (scope, pack))."""
    out = glass_placement()
    s = lib().glass_robo_placement(op, n, batch, ctypes.byref(out))
    return s, (out.scope, out.pack)


def glass_robo_feasible(op, n, scope, pack):
    return bool(lib().glass_robo_feasible(op, n, glass_placement(scope, pack)))


def glass_peak_probe(kind, iters, blocks, threads, sink, stream=None):
    """Launch one pipe-throughput probe; returns (status, flops of the launch)."""
    f = ctypes.c_double(0.0)
    st = lib().glass_peak_probe(kind, iters, blocks, threads, _ptr(sink), ctypes.byref(f), _stream(stream))
    return st, f.value


def glass_status_string(s):
    return status_string(s)


def glass_version():
    return lib().glass_version().decode()
