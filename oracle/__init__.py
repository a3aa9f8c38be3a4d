"""FP64 CPU oracle for the batched small-matrix operations (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``glass_oracle.c`` (plain loops, FP64), and
this module only marshals numpy arrays into it through ctypes.

Every array is a flat, C-contiguous numpy buffer laid out column-major per
problem, exactly as the device library stores its operands.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glass_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int)
_int = ctypes.c_int
_ll = ctypes.c_longlong


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        sig = {
            "oracle_set_threads": (None, [_int]),
            "oracle_max_threads": (_int, []),
            "oracle_gemm_f64": (None, [_int, _int, _int, _D, _int, _ll, _D, _int, _ll,
                                       _D, _int, _ll, _int]),
            "oracle_potrf_f64": (None, [_int, _D, _int, _ll, _I, _int]),
            "oracle_trsm_f64": (None, [_int, _int, _D, _int, _ll, _D, _int, _ll, _int]),
            "oracle_potrs_f64": (None, [_int, _int, _D, _int, _ll, _D, _int, _ll, _int]),
            "oracle_posv_f64": (None, [_int, _int, _D, _int, _ll, _D, _int, _ll, _I, _int]),
            "oracle_getrf_f64": (None, [_int, _D, _int, _ll, _I, _I, _D, _int]),
            "oracle_getrf_f32": (None, [_int, _F, _int, _ll, _I, _I, _D, _int]),
            "oracle_getrs_f64": (None, [_int, _int, _D, _int, _ll, _I, _D, _int, _ll, _int]),
            "oracle_getrf_getrs_f64": (None, [_int, _int, _D, _int, _ll, _I, _D, _int, _ll,
                                              _I, _int]),
            "oracle_gemm_ex_f64": (None, [_int, _int, _int, _int, _int, ctypes.c_double, _D, _int, _ll, _D, _int,
                                          _ll, ctypes.c_double, _D, _int, _ll, _int]),
            "oracle_riccati_gain_f64": (None, [_int, _int, _D, _ll, _D, _ll, _D, _ll, _D, _ll, _D, _ll, _I,
                                               _int]),
            "oracle_quat_retract_f64": (None, [_D, _D, _D, _int]),
            "oracle_quat_error_f64": (None, [_D, _D, _D, _int]),
            "oracle_se3_retract_f64": (None, [_D, _D, _D, _int]),
            "oracle_motion_cross_f64": (None, [_D, _D, _D, _int]),
            "oracle_eig3_f64": (None, [_D, _D, _D, _int]),
            "oracle_svd3_f64": (None, [_D, _D, _D, _D, _int]),
            "oracle_closest_rotation_f64": (None, [_D, _D, _int]),
            "oracle_argmax_f64": (None, [_int, _D, _ll, _I, _int]),
            "oracle_softmax_f64": (None, [_int, _D, _ll, _D, _ll, _int]),
            "oracle_dot_f64": (None, [_int, _D, _ll, _D, _ll, _D, _int]),
            "oracle_gemv_f64": (None, [_int, _int, _int, ctypes.c_double, _D, _int, _ll, _D, _ll,
                                       ctypes.c_double, _D, _ll, _int]),
            "oracle_btd_matvec_f64": (None, [_int, _int, _D, _D, _D, _D, _int]),
            "oracle_btd_posv_f64": (None, [_int, _int, _D, _D, _D, _I, _int]),
            "oracle_btd_pcg_f64": (None, [_int, _int, _D, _D, _D, _D, _int, ctypes.c_double, _I, _int]),
            "oracle_rot3_compose_f64": (None, [_int, _D, _ll, _D, _ll, _int]),
            "oracle_se3_apply_f64": (None, [_int, _D, _ll, _int, _D, _ll, _D, _ll, _int]),
            "oracle_mlp_nparams": (_ll, [_int, _int, _int]),
            "oracle_mlp_fwd_f64": (None, [_int, _int, _int, _D, _int, _D, _D, _D, _D]),
            "oracle_mlp_loss_grad_f64": (ctypes.c_double, [_int, _int, _int, _D, _int, _D,
                                                           _D, _D, _D]),
            "oracle_adam_step_f64": (None, [_ll, _D, _D, _D, _D, _int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _fp(a):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(_F)


def _ip(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64).copy()


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# ---------------------------------------------------------------- operations
def gemm(m, n, k, A, B, batch, lda=None, ldb=None, ldc=None, sA=None, sB=None, sC=None):
    lda = m if lda is None else lda
    ldb = k if ldb is None else ldb
    ldc = m if ldc is None else ldc
    sA = lda * k if sA is None else sA
    sB = ldb * n if sB is None else sB
    sC = ldc * n if sC is None else sC
    A = _f64(A)
    B = _f64(B)
    C = np.zeros(max(1, sC * batch), dtype=np.float64)
    _load().oracle_gemm_f64(m, n, k, _dp(A), lda, sA, _dp(B), ldb, sB, _dp(C), ldc, sC, batch)
    return C


def potrf(n, A, batch, lda=None, sA=None):
    lda = n if lda is None else lda
    sA = lda * n if sA is None else sA
    L = _f64(A)
    info = np.zeros(max(1, batch), dtype=np.int32)
    _load().oracle_potrf_f64(n, _dp(L), lda, sA, _ip(info), batch)
    return L, info[:batch]


def trsm(n, nrhs, L, B, batch, lda=None, sA=None, ldb=None, sB=None):
    lda = n if lda is None else lda
    sA = lda * n if sA is None else sA
    ldb = n if ldb is None else ldb
    sB = ldb * nrhs if sB is None else sB
    X = _f64(B)
    _load().oracle_trsm_f64(n, nrhs, _dp(_f64(L)), lda, sA, _dp(X), ldb, sB, batch)
    return X


def potrs(n, nrhs, L, B, batch, lda=None, sA=None, ldb=None, sB=None):
    lda = n if lda is None else lda
    sA = lda * n if sA is None else sA
    ldb = n if ldb is None else ldb
    sB = ldb * nrhs if sB is None else sB
    X = _f64(B)
    _load().oracle_potrs_f64(n, nrhs, _dp(_f64(L)), lda, sA, _dp(X), ldb, sB, batch)
    return X


def posv(n, nrhs, A, B, batch, lda=None, sA=None, ldb=None, sB=None):
    lda = n if lda is None else lda
    sA = lda * n if sA is None else sA
    ldb = n if ldb is None else ldb
    sB = ldb * nrhs if sB is None else sB
    L = _f64(A)
    X = _f64(B)
    info = np.zeros(max(1, batch), dtype=np.int32)
    _load().oracle_posv_f64(n, nrhs, _dp(L), lda, sA, _dp(X), ldb, sB, _ip(info), batch)
    return L, X, info[:batch]


def getrf(n, A, batch, lda=None, sA=None, precision="f64"):
    """Returns (LU, ipiv[batch*n], info[batch], gap[batch])."""
    lda = n if lda is None else lda
    sA = lda * n if sA is None else sA
    ipiv = np.zeros(max(1, batch * n), dtype=np.int32)
    info = np.zeros(max(1, batch), dtype=np.int32)
    gap = np.zeros(max(1, batch), dtype=np.float64)
    if precision == "f64":
        LU = _f64(A)
        _load().oracle_getrf_f64(n, _dp(LU), lda, sA, _ip(ipiv), _ip(info), _dp(gap), batch)
    elif precision == "f32":
        LU = np.ascontiguousarray(A, dtype=np.float32).copy()
        _load().oracle_getrf_f32(n, _fp(LU), lda, sA, _ip(ipiv), _ip(info), _dp(gap), batch)
    else:
        raise ValueError(precision)
    return LU, ipiv[:batch * n], info[:batch], gap[:batch]


def getrs(n, nrhs, LU, ipiv, B, batch, lda=None, sA=None, ldb=None, sB=None):
    lda = n if lda is None else lda
    sA = lda * n if sA is None else sA
    ldb = n if ldb is None else ldb
    sB = ldb * nrhs if sB is None else sB
    X = _f64(B)
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _load().oracle_getrs_f64(n, nrhs, _dp(_f64(LU)), lda, sA, _ip(piv), _dp(X), ldb, sB, batch)
    return X


def getrf_getrs(n, nrhs, A, B, batch, lda=None, sA=None, ldb=None, sB=None):
    lda = n if lda is None else lda
    sA = lda * n if sA is None else sA
    ldb = n if ldb is None else ldb
    sB = ldb * nrhs if sB is None else sB
    LU = _f64(A)
    X = _f64(B)
    ipiv = np.zeros(max(1, batch * n), dtype=np.int32)
    info = np.zeros(max(1, batch), dtype=np.int32)
    _load().oracle_getrf_getrs_f64(n, nrhs, _dp(LU), lda, sA, _ip(ipiv), _dp(X), ldb, sB,
                                   _ip(info), batch)
    return LU, ipiv[:batch * n], X, info[:batch]


def gemm_ex(ta, tb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch):
    """C = alpha op(A) op(B) + beta C (returns the new C; C may be None when beta == 0)."""
    A, B = _f64(A), _f64(B)
    C = np.zeros(max(1, sC * batch), dtype=np.float64) if C is None else _f64(C)
    _load().oracle_gemm_ex_f64(int(bool(ta)), int(bool(tb)), m, n, k, float(alpha), _dp(A), lda, sA, _dp(B), ldb,
                               sB, float(beta), _dp(C), ldc, sC, batch)
    return C


def riccati_gain(nx, nu, A, B, P, R, batch, sA=None, sB=None, sP=None, sR=None, sK=None):
    """K = (R + B^T P B)^{-1} B^T P A per problem; returns (K, info)."""
    sA = nx * nx if sA is None else sA
    sB = nx * nu if sB is None else sB
    sP = nx * nx if sP is None else sP
    sR = nu * nu if sR is None else sR
    sK = nu * nx if sK is None else sK
    A, B, P, R = _f64(A), _f64(B), _f64(P), _f64(R)
    K = np.zeros(max(1, sK * batch), dtype=np.float64)
    info = np.zeros(max(1, batch), dtype=np.int32)
    _load().oracle_riccati_gain_f64(nx, nu, _dp(A), sA, _dp(B), sB, _dp(P), sP, _dp(R), sR, _dp(K), sK, _ip(info),
                                    batch)
    return K, info[:batch]


# ------------------------------------------------ robotics operations
def _out(n):
    return np.zeros(max(1, n), dtype=np.float64)


def quat_retract(q, d, batch):
    """q * Exp(d), q = (w, x, y, z) [batch][4], d [batch][3] -> [batch][4]."""
    o = _out(4 * batch)
    _load().oracle_quat_retract_f64(_dp(_f64(q)), _dp(_f64(d)), _dp(o), batch)
    return o


def quat_error(q1, q2, batch):
    """Log(conj(q1) * q2) -> [batch][3]."""
    o = _out(3 * batch)
    _load().oracle_quat_error_f64(_dp(_f64(q1)), _dp(_f64(q2)), _dp(o), batch)
    return o


def se3_retract(T, xi, batch):
    """T Exp(xi), T 4x4 column-major [batch][16], xi = (rho, phi) [batch][6]."""
    o = _out(16 * batch)
    _load().oracle_se3_retract_f64(_dp(_f64(T)), _dp(_f64(xi)), _dp(o), batch)
    return o


def motion_cross(v, m, batch):
    """v x m for motion vectors (linear, angular) [batch][6]."""
    o = _out(6 * batch)
    _load().oracle_motion_cross_f64(_dp(_f64(v)), _dp(_f64(m)), _dp(o), batch)
    return o


def eig3(A, batch):
    """(w [batch][3] ascending, V [batch][9] column-major eigenvectors)."""
    w, V = _out(3 * batch), _out(9 * batch)
    _load().oracle_eig3_f64(_dp(_f64(A)), _dp(w), _dp(V), batch)
    return w, V


def svd3(M, batch):
    """(U [batch][9], s [batch][3] descending, V [batch][9])."""
    U, sv, V = _out(9 * batch), _out(3 * batch), _out(9 * batch)
    _load().oracle_svd3_f64(_dp(_f64(M)), _dp(U), _dp(sv), _dp(V), batch)
    return U, sv, V


def closest_rotation(M, batch):
    o = _out(9 * batch)
    _load().oracle_closest_rotation_f64(_dp(_f64(M)), _dp(o), batch)
    return o


def argmax(n, x, batch, sx=None):
    sx = n if sx is None else sx
    idx = np.zeros(max(1, batch), dtype=np.int32)
    _load().oracle_argmax_f64(n, _dp(_f64(x)), sx, _ip(idx), batch)
    return idx[:batch]


def softmax(n, x, batch, sx=None):
    sx = n if sx is None else sx
    y = _out(n * batch)
    _load().oracle_softmax_f64(n, _dp(_f64(x)), sx, _dp(y), n, batch)
    return y


# ------------------------------------------------ BLAS-1/2, block-tridiagonal
def dot(n, x, y, batch, sx=None, sy=None):
    sx = n if sx is None else sx
    sy = n if sy is None else sy
    out = _out(batch)
    _load().oracle_dot_f64(n, _dp(_f64(x)), sx, _dp(_f64(y)), sy, _dp(out), batch)
    return out[:batch]


def gemv(trans, m, n, alpha, A, lda, sA, x, sx, beta, y, sy, batch):
    """y = alpha op(A) x + beta y; returns the new y (y may be None when beta == 0)."""
    y = np.zeros(max(1, sy * batch), dtype=np.float64) if y is None else _f64(y)
    _load().oracle_gemv_f64(int(bool(trans)), m, n, float(alpha), _dp(_f64(A)), lda, sA, _dp(_f64(x)), sx,
                            float(beta), _dp(y), sy, batch)
    return y


def btd_matvec(nb, N, D, O, x, batch):
    """y = T x, T symmetric block-tridiagonal (D: [batch][N][nb*nb], O: [batch][N-1][nb*nb])."""
    y = _out(N * nb * batch)
    _load().oracle_btd_matvec_f64(nb, N, _dp(_f64(D)), _dp(_f64(O) if N > 1 else np.zeros(1)), _dp(_f64(x)),
                                  _dp(y), batch)
    return y


def btd_posv(nb, N, D, O, b, batch):
    """(x, info) with T x = b by the dense Cholesky solve of the assembled T."""
    x = _f64(b)
    info = np.zeros(max(1, batch), dtype=np.int32)
    _load().oracle_btd_posv_f64(nb, N, _dp(_f64(D)), _dp(_f64(O) if N > 1 else np.zeros(1)), _dp(x), _ip(info),
                                batch)
    return x, info[:batch]


def btd_pcg(nb, N, D, O, b, x0, iters, tol, batch):
    """Block-Jacobi PCG on the block-tridiagonal T: (x, iters_done)."""
    x = _f64(x0)
    done = np.zeros(max(1, batch), dtype=np.int32)
    _load().oracle_btd_pcg_f64(nb, N, _dp(_f64(D)), _dp(_f64(O)), _dp(_f64(b)), _dp(x), int(iters), float(tol),
                               _ip(done), batch)
    return x, done[:batch]


def rot3_compose(chain, Rs, batch, sRs=None, sR=9):
    sRs = 9 * chain if sRs is None else sRs
    R = np.zeros(max(1, sR * batch), dtype=np.float64)
    _load().oracle_rot3_compose_f64(chain, _dp(_f64(Rs)), sRs, _dp(R), sR, batch)
    return R


def se3_apply(chain, T, npts, P, batch, sT=None, sP=None, sQ=None):
    sT = 16 * chain if sT is None else sT
    sP = 3 * npts if sP is None else sP
    sQ = 3 * npts if sQ is None else sQ
    Q = np.zeros(max(1, sQ * batch), dtype=np.float64)
    _load().oracle_se3_apply_f64(chain, _dp(_f64(T)), sT, npts, _dp(_f64(P)), sP, _dp(Q),
                                 sQ, batch)
    return Q


# ---------------------------------------------------------------- cost model
def mlp_nparams(din, h, dout):
    return int(_load().oracle_mlp_nparams(din, h, dout))


def mlp_fwd(din, h, dout, w, X):
    X = _f64(X)
    rows = X.size // din
    Y = np.zeros(rows * dout, dtype=np.float64)
    _load().oracle_mlp_fwd_f64(din, h, dout, _dp(_f64(w)), rows, _dp(X), _dp(Y), None, None)
    return Y.reshape(rows, dout)


def mlp_loss_grad(din, h, dout, w, X, T, M):
    X = _f64(X)
    rows = X.size // din
    g = np.zeros(mlp_nparams(din, h, dout), dtype=np.float64)
    loss = _load().oracle_mlp_loss_grad_f64(din, h, dout, _dp(_f64(w)), rows, _dp(X),
                                            _dp(_f64(T)), _dp(_f64(M)), _dp(g))
    return float(loss), g


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on w, m, v (float64 contiguous arrays)."""
    _load().oracle_adam_step_f64(w.size, _dp(w), _dp(_f64(g)), _dp(m), _dp(v), int(t), lr,
                                 b1, b2, eps)
