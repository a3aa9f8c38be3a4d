"""FP64 storage variants (gemm, potrf/potrs/posv, trsm, getrf+getrs) on the
GPU, through the C ABI (opts.dtype = GLASS_F64), against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
BATCH = 133


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


def _dev(x, dtype=np.float64):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _placements(op, n):
    """Thread scope up to n = 8; warp scope while the packed problems' shared
    memory (pack * n * (n | 1) doubles) fits the 227 KB of a CTA."""
    out = []
    for s, packs in ((g.GLASS_SCOPE_THREAD, (1, 4)), (g.GLASS_SCOPE_WARP, (1, 2, 8))):
        for p in packs:
            if s == g.GLASS_SCOPE_THREAD and n > 8:
                continue
            if s == g.GLASS_SCOPE_WARP and op != g.GLASS_OP_GEMM and p * n * (n | 1) * 8 + p * 256 > 227 * 1024:
                continue
            out.append((s, p))
    return out + [(g.GLASS_SCOPE_AUTO, 0)]


def test_infeasible_f64_placements_are_refused():
    o = g.make_opts(dtype=g.GLASS_F64, scope=g.GLASS_SCOPE_WARP, pack=8)
    A, B = _dev(np.eye(64).reshape(-1).repeat(1)), _dev(np.zeros(64))
    info = _dev(np.zeros(1, np.int32), np.int32)
    assert g.glass_batched_posv(64, 1, A, 64, 4096, B, 64, 64, info, 1, o) == g.GLASS_ERR_INVALID_VALUE
    o = g.make_opts(dtype=g.GLASS_F64, scope=g.GLASS_SCOPE_THREAD, pack=1)
    assert g.glass_batched_posv(12, 1, A, 12, 144, B, 12, 12, info, 1, o) == g.GLASS_ERR_INVALID_VALUE


def _o(s, p):
    return g.make_opts(dtype=g.GLASS_F64, scope=s, pack=p)


@pytest.mark.parametrize("m,n,k", [(3, 3, 3), (7, 5, 6), (8, 8, 8), (24, 24, 24), (33, 17, 40), (64, 64, 64)])
def test_gemm_f64(m, n, k):
    r = W.rng(400 + m + n + k)
    lda, ldb, ldc = m + 1, k + 2, m + 3
    A = r.standard_normal(BATCH * lda * k)
    B = r.standard_normal(BATCH * ldb * n)
    ref = oracle.gemm(m, n, k, A, B, BATCH, lda=lda, ldb=ldb, ldc=ldc, sA=lda * k, sB=ldb * n, sC=ldc * n)
    absr = oracle.gemm(m, n, k, np.abs(A), np.abs(B), BATCH, lda=lda, ldb=ldb, ldc=ldc, sA=lda * k, sB=ldb * n,
                       sC=ldc * n)
    for s, p in _placements(g.GLASS_OP_GEMM, max(m, n, k)):
        dC = _dev(np.full(BATCH * ldc * n, 7.0))
        g.check(g.glass_batched_gemm(m, n, k, _dev(A), lda, lda * k, _dev(B), ldb, ldb * n, dC, ldc, ldc * n, BATCH,
                                     _o(s, p)), f"gemm f64 {s}x{p}")
        got = _host(dC).reshape(BATCH, n, ldc)
        want, bound = ref.reshape(BATCH, n, ldc), absr.reshape(BATCH, n, ldc)
        assert (np.abs(got[:, :, :m] - want[:, :, :m]) <= 2 * k * U64 * bound[:, :, :m] + 1e-300).all(), (s, p)
        assert (got[:, :, m:] == 7.0).all()


@pytest.mark.parametrize("n", [1, 3, 5, 8, 12, 33, 64])
def test_posv_potrf_potrs_f64(n):
    A = W.spd(n, BATCH, 410 + n).astype(np.float64)
    Bm = W.rng(411 + n).standard_normal(BATCH * n * 2)
    L_ref, X_ref, info_ref = oracle.posv(n, 2, A, Bm, BATCH)
    for s, p in _placements(g.GLASS_OP_POSV, n):
        dA, dB = _dev(A), _dev(Bm)
        info = _dev(np.full(BATCH, -3, np.int32), np.int32)
        g.check(g.glass_batched_posv(n, 2, dA, n, n * n, dB, n, 2 * n, info, BATCH, _o(s, p)), f"posv f64 {s}x{p}")
        assert (_host(info) == 0).all()
        X = _host(dB)
        assert np.abs(X - X_ref).max() <= 1e-12 * np.abs(X_ref).max() * max(1, n / 8), (n, s, p)
        Lg = np.tril(W.from_colmajor(_host(dA), BATCH, n, n))
        assert np.abs(Lg - np.tril(W.from_colmajor(L_ref, BATCH, n, n))).max() <= 1e-12 * np.abs(L_ref).max()
        up = np.triu_indices(n, 1)
        assert np.array_equal(W.from_colmajor(_host(dA), BATCH, n, n)[:, up[0], up[1]],
                              W.from_colmajor(A, BATCH, n, n)[:, up[0], up[1]])
        # split calls
        dA2, dB2 = _dev(A), _dev(Bm)
        g.check(g.glass_batched_potrf(n, dA2, n, n * n, info, BATCH, _o(s, p)))
        g.check(g.glass_batched_potrs(n, 2, dA2, n, n * n, dB2, n, 2 * n, BATCH, _o(s, p)))
        assert np.abs(_host(dB2) - X_ref).max() <= 1e-12 * np.abs(X_ref).max() * max(1, n / 8)


@pytest.mark.parametrize("n", [2, 6, 16, 40, 64])
def test_cholesky_f64_integer_exact_and_info(n):
    A, L0 = W.int_cholesky_factor(n, 40, 420 + n)
    X0 = W.int_matrix(n, 2, 40, 421 + n, -3, 3)
    Bc = W.colmajor(A @ X0, dtype=np.float64)
    for s, p in _placements(g.GLASS_OP_POSV, n):
        dA, dB = _dev(W.colmajor(A, dtype=np.float64)), _dev(Bc)
        info = _dev(np.zeros(40, np.int32), np.int32)
        g.check(g.glass_batched_posv(n, 2, dA, n, n * n, dB, n, 2 * n, info, 40, _o(s, p)))
        assert np.array_equal(np.tril(W.from_colmajor(_host(dA), 40, n, n)), L0), (n, s, p)
        assert np.array_equal(W.from_colmajor(_host(dB), 40, n, 2), X0), (n, s, p)
    # a non-SPD matrix reports its failing column
    Abad = A.copy()
    j = n // 2
    Abad[:, j, j] -= L0[:, j, j] ** 2 + 1.0
    info = _dev(np.zeros(40, np.int32), np.int32)
    g.check(g.glass_batched_potrf(n, _dev(W.colmajor(Abad, dtype=np.float64)), n, n * n, info, 40,
                                  _o(g.GLASS_SCOPE_AUTO, 0)))
    assert (_host(info) == j + 1).all()


@pytest.mark.parametrize("n", [4, 8, 17, 64])
def test_trsm_f64_integer_exact(n):
    L = W.int_lower_pow2_diag(n, 40, 430 + n)
    X0 = W.int_matrix(n, 5, 40, 431 + n, -3, 3)
    B = W.colmajor(L @ X0, dtype=np.float64)
    Lg = L.copy()
    Lg[:, np.triu_indices(n, 1)[0], np.triu_indices(n, 1)[1]] = np.nan   # upper never read
    for s, p in _placements(g.GLASS_OP_TRSM, n):
        dB = _dev(B)
        g.check(g.glass_batched_trsm(n, 5, _dev(W.colmajor(Lg, dtype=np.float64)), n, n * n, dB, n, n * 5, 40,
                                     _o(s, p)))
        assert np.array_equal(W.from_colmajor(_host(dB), 40, n, 5), X0), (n, s, p)


@pytest.mark.parametrize("n", [1, 3, 7, 8, 12, 33, 64])
def test_getrf_getrs_f64(n):
    A = W.gaussian(BATCH * n * n, 440 + n).astype(np.float64)
    B = W.gaussian(BATCH * n, 441 + n).astype(np.float64)
    LU_ref, piv_ref, X_ref, info_ref = oracle.getrf_getrs(n, 1, A, B, BATCH)
    _, _, _, gap = oracle.getrf(n, A, BATCH)
    clear = gap >= 1e-9
    cond = np.linalg.cond(W.from_colmajor(A, BATCH, n, n))
    for s, p in _placements(g.GLASS_OP_GETRF_GETRS, n):
        dA, dB = _dev(A), _dev(B)
        ipiv = _dev(np.zeros(BATCH * n, np.int32), np.int32)
        info = _dev(np.full(BATCH, -3, np.int32), np.int32)
        g.check(g.glass_batched_getrf_getrs(n, 1, dA, n, n * n, ipiv, dB, n, n, info, BATCH, _o(s, p)),
                f"lu f64 {s}x{p}")
        assert np.array_equal(_host(info), info_ref)
        pv = _host(ipiv).reshape(BATCH, n)
        assert np.array_equal(pv[clear], piv_ref.reshape(BATCH, n)[clear]), (n, s, p)
        ok = clear & (info_ref == 0) & (cond < 1e6)
        X = _host(dB).reshape(BATCH, n)
        Xr = X_ref.reshape(BATCH, n)
        scale = np.abs(Xr[ok]).max(axis=1, keepdims=True)
        assert (np.abs(X[ok] - Xr[ok]) <= 1e-9 * scale).all(), (n, s, p)


@pytest.mark.parametrize("n", [2, 6, 12, 64])
def test_getrf_f64_dyadic_bit_exact(n):
    A, perm, L0, U0 = W.dyadic_lu(n, 30, 450 + n)
    for s, p in _placements(g.GLASS_OP_GETRF_GETRS, n):
        dA = _dev(W.colmajor(A, dtype=np.float64))
        ipiv = _dev(np.zeros(30 * n, np.int32), np.int32)
        info = _dev(np.zeros(30, np.int32), np.int32)
        g.check(g.glass_batched_getrf_getrs(n, 0, dA, n, n * n, ipiv, None, n, n, info, 30, _o(s, p)))
        LU = W.from_colmajor(_host(dA), 30, n, n)
        pv = _host(ipiv).reshape(30, n)
        for b in range(30):
            perm_b = np.arange(n)
            for j in range(n):
                perm_b[[j, pv[b, j]]] = perm_b[[pv[b, j], j]]
            assert np.array_equal(perm_b, perm[b]), (n, s, p)
            assert np.array_equal(np.tril(LU[b], -1) + np.eye(n), L0[b]), (n, s, p)
            assert np.array_equal(np.triu(LU[b]), U0[b]), (n, s, p)
