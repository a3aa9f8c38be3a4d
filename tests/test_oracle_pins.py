"""Pins of the FP64 oracle against what mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: SciPy/NumPy
library routines, hand-worked examples (tests/golden), exact-integer and
dyadic constructions whose factors are known without factorizing, closed
forms, and brute force on tiny inputs.  A plausible slip in the oracle (a
dropped term, a wrong index, a transposed operand, a wrong pivot rule) fails
at least one of them.
"""
from fractions import Fraction
import itertools
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2609_28179_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(Fraction(v)) for v in vals]
    return out


def _cm(mats):
    return W.colmajor(np.asarray(mats, dtype=np.float64), dtype=np.float64)


def _mats(flat, batch, r, c):
    return W.from_colmajor(flat, batch, r, c)


# ----------------------------------------------------------------- golden
def test_golden_cholesky_3x3():
    g = _golden("cholesky_3x3.txt")
    A = np.array(g["A"]).reshape(3, 3)
    L, info = oracle.potrf(3, _cm([A]), 1)
    assert info[0] == 0
    Lm = np.tril(_mats(L, 1, 3, 3)[0])
    assert np.array_equal(Lm, np.array(g["L"]).reshape(3, 3))
    _, X, info = oracle.posv(3, 1, _cm([A]), np.array(g["b"]), 1)
    np.testing.assert_allclose(X, g["x"], rtol=0, atol=1e-15)


def test_golden_lu_3x3():
    g = _golden("lu_3x3.txt")
    A = np.array(g["A"]).reshape(3, 3)
    LU, ipiv, info, _ = oracle.getrf(3, _cm([A]), 1)
    assert info[0] == 0
    assert list(ipiv) == [int(v) for v in g["ipiv"]]
    np.testing.assert_allclose(_mats(LU, 1, 3, 3)[0], np.array(g["LU"]).reshape(3, 3),
                               rtol=0, atol=1e-15)
    _, _, X, _ = oracle.getrf_getrs(3, 1, _cm([A]), np.array(g["b"]), 1)
    np.testing.assert_allclose(X, g["x"], rtol=0, atol=1e-14)


# ------------------------------------------------------------------- gemm
@pytest.mark.parametrize("m,n,k", [(3, 3, 3), (7, 5, 6), (64, 64, 64), (1, 9, 2)])
def test_gemm_vs_numpy(m, n, k):
    g = W.rng(1)
    b = 5
    A = g.standard_normal((b, m, k))
    B = g.standard_normal((b, k, n))
    C = oracle.gemm(m, n, k, _cm(A), _cm(B), b)
    np.testing.assert_allclose(_mats(C, b, m, n), A @ B, rtol=1e-12, atol=1e-12)


def test_gemm_integer_exact_and_structure():
    n, b = 64, 3
    A = W.int_matrix(n, n, b, 2)
    B = W.int_matrix(n, n, b, 3)
    C = oracle.gemm(n, n, n, _cm(A), _cm(B), b)
    assert np.array_equal(_mats(C, b, n, n), A @ B)
    # identity on the left, permutation on the right
    I = np.broadcast_to(np.eye(n), (b, n, n))
    C = oracle.gemm(n, n, n, _cm(I), _cm(B), b)
    assert np.array_equal(_mats(C, b, n, n), B)
    perm = W.rng(4).permutation(n)
    P = np.eye(n)[:, perm][None].repeat(b, 0)
    C = oracle.gemm(n, n, n, _cm(A), _cm(P), b)
    assert np.array_equal(_mats(C, b, n, n), A[:, :, perm])


def test_gemm_strided_leading_dims():
    # padded lda/ldb/ldc and batch strides larger than the matrix
    m, n, k, b = 5, 4, 3, 2
    g = W.rng(5)
    lda, ldb, ldc = 7, 6, 9
    A = g.standard_normal(b * lda * k + 11)
    B = g.standard_normal(b * ldb * n + 13)
    C = oracle.gemm(m, n, k, A, B, b, lda=lda, ldb=ldb, ldc=ldc,
                    sA=lda * k + 11 // b, sB=ldb * n + 13 // b, sC=ldc * n + 1)
    for bb in range(b):
        a = A[bb * (lda * k + 5):][: lda * k].reshape(k, lda).T[:m]
        bm = B[bb * (ldb * n + 6):][: ldb * n].reshape(n, ldb).T[:k]
        c = C[bb * (ldc * n + 1):][: ldc * n].reshape(n, ldc).T[:m]
        np.testing.assert_allclose(c, a @ bm, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ potrf
@pytest.mark.parametrize("n", [1, 2, 3, 6, 7, 12, 24, 64])
def test_potrf_vs_scipy(n):
    b = 4
    A = _mats(W.spd(n, b, 10 + n).astype(np.float64), b, n, n)
    L, info = oracle.potrf(n, _cm(A), b)
    assert (info == 0).all()
    Lm = np.tril(_mats(L, b, n, n))
    for i in range(b):
        ref = sla.cholesky(A[i], lower=True)
        np.testing.assert_allclose(Lm[i], ref, rtol=1e-12, atol=1e-12)


def test_potrf_leaves_upper_untouched():
    n = 6
    A = _mats(W.spd(n, 1, 3).astype(np.float64), 1, n, n)[0].copy()
    A[np.triu_indices(n, 1)] = 12345.0
    L, info = oracle.potrf(n, _cm([A]), 1)
    Lm = _mats(L, 1, n, n)[0]
    assert info[0] == 0
    assert (Lm[np.triu_indices(n, 1)] == 12345.0).all()


@pytest.mark.parametrize("n", [2, 5, 16, 64])
def test_potrf_integer_exact(n):
    A, L0 = W.int_cholesky_factor(n, 6, 20 + n)
    L, info = oracle.potrf(n, _cm(A), 6)
    assert (info == 0).all()
    assert np.array_equal(np.tril(_mats(L, 6, n, n)), L0)


def test_potrf_2x2_closed_form():
    g = W.rng(7)
    for _ in range(20):
        M = g.standard_normal((2, 2))
        A = M @ M.T + 0.5 * np.eye(2)
        L, info = oracle.potrf(2, _cm([A]), 1)
        l11 = np.sqrt(A[0, 0])
        l21 = A[1, 0] / l11
        l22 = np.sqrt(A[1, 1] - l21 ** 2)
        Lm = _mats(L, 1, 2, 2)[0]
        np.testing.assert_allclose([Lm[0, 0], Lm[1, 0], Lm[1, 1]], [l11, l21, l22],
                                   rtol=1e-14)


@pytest.mark.parametrize("j", [0, 1, 4, 7])
def test_potrf_info_non_spd(j):
    n = 8
    A, L0 = W.int_cholesky_factor(n, 1, 30 + j)
    A = A[0].copy()
    A[j, j] -= L0[0, j, j] ** 2 + 1.0        # pivot at column j becomes -1
    L, info = oracle.potrf(n, _cm([A]), 1)
    assert info[0] == j + 1
    A[j, j] += 1.0                           # pivot exactly 0 is also a failure
    L, info = oracle.potrf(n, _cm([A]), 1)
    assert info[0] == j + 1
    A[j, j] = np.nan
    L, info = oracle.potrf(n, _cm([A]), 1)
    assert info[0] == j + 1


# ---------------------------------------------------------- trsm / potrs
@pytest.mark.parametrize("n,k", [(1, 1), (3, 2), (12, 12), (64, 5)])
def test_trsm_vs_scipy(n, k):
    b = 3
    g = W.rng(40 + n)
    L = np.tril(g.standard_normal((b, n, n))) + 3 * np.eye(n)
    B = g.standard_normal((b, n, k))
    X = oracle.trsm(n, k, _cm(L), _cm(B), b)
    Xm = _mats(X, b, n, k)
    for i in range(b):
        ref = sla.solve_triangular(L[i], B[i], lower=True)
        np.testing.assert_allclose(Xm[i], ref, rtol=1e-11, atol=1e-11)


def test_trsm_ignores_upper_triangle():
    n, k = 5, 2
    g = W.rng(41)
    L = np.tril(g.standard_normal((1, n, n))) + 3 * np.eye(n)
    Lg = L.copy()
    Lg[0][np.triu_indices(n, 1)] = np.nan
    B = g.standard_normal((1, n, k))
    np.testing.assert_array_equal(oracle.trsm(n, k, _cm(Lg), _cm(B), 1),
                                  oracle.trsm(n, k, _cm(L), _cm(B), 1))


@pytest.mark.parametrize("n", [1, 4, 17, 64])
def test_trsm_integer_exact(n):
    k, b = 3, 4
    L = W.int_lower_pow2_diag(n, b, 50 + n)
    X0 = W.int_matrix(n, k, b, 51 + n, -3, 3)
    B = L @ X0
    X = oracle.trsm(n, k, _cm(L), _cm(B), b)
    assert np.array_equal(_mats(X, b, n, k), X0)


@pytest.mark.parametrize("n", [2, 9, 32, 64])
def test_potrs_exact_and_vs_scipy(n):
    k, b = 2, 3
    L = W.int_lower_pow2_diag(n, b, 60 + n, positive=True)
    X0 = W.int_matrix(n, k, b, 61 + n, -3, 3)
    B = L @ np.transpose(L, (0, 2, 1)) @ X0
    X = oracle.potrs(n, k, _cm(L), _cm(B), b)
    assert np.array_equal(_mats(X, b, n, k), X0)
    A = _mats(W.spd(n, b, 62 + n).astype(np.float64), b, n, n)
    Bg = W.rng(63).standard_normal((b, n, k))
    Lf, info = oracle.potrf(n, _cm(A), b)
    X = oracle.potrs(n, k, Lf, _cm(Bg), b)
    for i in range(b):
        ref = sla.cho_solve((sla.cholesky(A[i], lower=True), True), Bg[i])
        np.testing.assert_allclose(_mats(X, b, n, k)[i], ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n", [6, 33, 64])
def test_posv_residual_and_factor(n):
    b, k = 5, 4
    A = _mats(W.spd(n, b, 70 + n).astype(np.float64), b, n, n)
    B = W.rng(71).standard_normal((b, n, k))
    L, X, info = oracle.posv(n, k, _cm(A), _cm(B), b)
    assert (info == 0).all()
    Lm = np.tril(_mats(L, b, n, n))
    Xm = _mats(X, b, n, k)
    np.testing.assert_allclose(Lm @ np.transpose(Lm, (0, 2, 1)), A, rtol=1e-12, atol=1e-10)
    res = np.abs(A @ Xm - B).max() / (np.abs(A).sum(-1).max() * np.abs(Xm).max())
    assert res < 1e-14


# ------------------------------------------------------------------ getrf
def _lu_unpack(LUm):
    n = LUm.shape[-1]
    L = np.tril(LUm, -1) + np.eye(n)
    U = np.triu(LUm)
    return L, U


def _perm_from_ipiv(ipiv, n):
    perm = np.arange(n)
    for j in range(n):
        p = ipiv[j]
        perm[[j, p]] = perm[[p, j]]
    return perm


@pytest.mark.parametrize("n", [1, 2, 3, 7, 14, 32, 64])
def test_getrf_vs_scipy(n):
    b = 4
    A = _mats(W.rng(80 + n).standard_normal(b * n * n), b, n, n)
    LU, ipiv, info, gap = oracle.getrf(n, _cm(A), b)
    assert (info == 0).all()
    for i in range(b):
        lu, piv = sla.lu_factor(A[i])
        assert np.array_equal(piv, ipiv[i * n:(i + 1) * n])
        np.testing.assert_allclose(_mats(LU, b, n, n)[i], lu, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("n", [2, 6, 12, 24, 64])
def test_getrf_dyadic_exact(n):
    b = 5
    A, perm, L0, U0 = W.dyadic_lu(n, b, 90 + n)
    for prec in ("f64", "f32"):
        LU, ipiv, info, gap = oracle.getrf(n, _cm(A), b, precision=prec)
        assert (info == 0).all()
        LUm = _mats(LU, b, n, n)
        for i in range(b):
            assert np.array_equal(_perm_from_ipiv(ipiv[i * n:(i + 1) * n], n), perm[i])
            L, U = _lu_unpack(LUm[i])
            assert np.array_equal(L, L0[i]) and np.array_equal(U, U0[i])
        assert (gap >= 0.5).all()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_getrf_brute_force_tiny(n):
    """Enumerate every row order; partial pivoting is the unique order whose
    unpivoted LU has all |l_ij| <= 1 (inputs are generic)."""
    g = W.rng(100 + n)
    for _ in range(25):
        A = g.standard_normal((n, n))
        winners = []
        for perm in itertools.permutations(range(n)):
            Ap = A[list(perm)]
            # Doolittle, closed form for n <= 3
            U = np.zeros((n, n))
            L = np.eye(n)
            for i in range(n):
                for j in range(i, n):
                    U[i, j] = Ap[i, j] - L[i, :i] @ U[:i, j]
                for j in range(i + 1, n):
                    L[j, i] = (Ap[j, i] - L[j, :i] @ U[:i, i]) / U[i, i]
            if np.abs(np.tril(L, -1)).max(initial=0.0) <= 1.0:
                winners.append((perm, L, U))
        assert len(winners) == 1
        perm, L0, U0 = winners[0]
        LU, ipiv, info, _ = oracle.getrf(n, _cm([A]), 1)
        assert tuple(_perm_from_ipiv(ipiv, n)) == perm
        L, U = _lu_unpack(_mats(LU, 1, n, n)[0])
        np.testing.assert_allclose(L, L0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(U, U0, rtol=1e-12, atol=1e-12)


def test_getrf_tie_takes_smallest_row_and_singular_info():
    # column 0 has equal magnitudes at rows 1 and 2: row 1 must win
    A = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [3.0, 0.0, 2.0]])
    _, ipiv, info, gap = oracle.getrf(3, _cm([A]), 1)
    assert ipiv[0] == 1 and info[0] == 0 and gap[0] == 0.0
    # exactly singular: second column is a multiple of the first
    A = np.array([[1.0, 2.0, 1.0], [2.0, 4.0, 0.0], [4.0, 8.0, 3.0]])
    _, ipiv, info, _ = oracle.getrf(3, _cm([A]), 1)
    assert info[0] == 2


@pytest.mark.parametrize("n", [3, 12, 64])
def test_getrs_vs_scipy(n):
    b, k = 3, 3
    A = _mats(W.general(n, b, 110 + n).astype(np.float64), b, n, n)
    B = W.rng(111).standard_normal((b, n, k))
    LU, ipiv, X, info = oracle.getrf_getrs(n, k, _cm(A), _cm(B), b)
    for i in range(b):
        ref = sla.lu_solve(sla.lu_factor(A[i]), B[i])
        np.testing.assert_allclose(_mats(X, b, n, k)[i], ref, rtol=1e-10, atol=1e-12)
    # split path gives the same answer
    LU2, ipiv2, info2, _ = oracle.getrf(n, _cm(A), b)
    X2 = oracle.getrs(n, k, LU2, ipiv2, _cm(B), b)
    np.testing.assert_array_equal(X, X2)


# -------------------------------------------------------------- geometry
def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def test_rot3_rz_addition():
    g = W.rng(120)
    for _ in range(10):
        a, b = g.uniform(-np.pi, np.pi, 2)
        R = oracle.rot3_compose(2, _cm([_rz(a), _rz(b)]), 1)
        np.testing.assert_allclose(_mats(R, 1, 3, 3)[0], _rz(a + b), atol=1e-14)


@pytest.mark.parametrize("chain", [1, 2, 3, 7, 64])
def test_rot3_chain_orthonormal_and_order(chain):
    b = 6
    Rs = W.rotations(b * chain, 121 + chain).astype(np.float64)
    R = _mats(oracle.rot3_compose(chain, Rs, b), b, 3, 3)
    mats = _mats(Rs, b * chain, 3, 3).reshape(b, chain, 3, 3)
    for i in range(b):
        ref = np.eye(3)
        for c in range(chain):
            ref = ref @ mats[i, c]
        np.testing.assert_allclose(R[i], ref, atol=1e-12)
        np.testing.assert_allclose(R[i].T @ R[i], np.eye(3), atol=1e-6)
        assert abs(np.linalg.det(R[i]) - 1.0) < 1e-6
    if chain >= 2:  # order matters: R0 R1 != R1 R0 in general
        swapped = mats[:, [1, 0] + list(range(2, chain))]
        R2 = _mats(oracle.rot3_compose(chain, _cm(swapped.reshape(-1, 3, 3)), b), b, 3, 3)
        assert np.abs(R2 - R).max() > 1e-3


def test_se3_inverse_identity_translation():
    b, npts = 4, 50
    T = W.se3_transforms(b, 130).astype(np.float64)
    P = W.gaussian(b * 3 * npts, 131).astype(np.float64)
    Q = oracle.se3_apply(1, T, npts, P, b)
    Tm = _mats(T, b, 4, 4)
    Tinv = np.zeros_like(Tm)
    for i in range(b):
        R, t = Tm[i, :3, :3], Tm[i, :3, 3]
        Ri = np.linalg.inv(R)   # inputs are FP32-rounded: R^T is not exact
        Tinv[i, :3, :3] = Ri
        Tinv[i, :3, 3] = -Ri @ t
        Tinv[i, 3, 3] = 1.0
    P2 = oracle.se3_apply(1, _cm(Tinv), npts, Q, b)
    np.testing.assert_allclose(P2, P, atol=1e-12)
    I = np.broadcast_to(np.eye(4), (b, 4, 4))
    np.testing.assert_array_equal(oracle.se3_apply(1, _cm(I), npts, P, b), P)
    Tt = np.broadcast_to(np.eye(4), (b, 4, 4)).copy()
    Tt[:, :3, 3] = [1.5, -2.0, 0.25]
    Qt = oracle.se3_apply(1, _cm(Tt), npts, P, b).reshape(b, npts, 3)
    np.testing.assert_allclose(Qt, P.reshape(b, npts, 3) + np.array([1.5, -2.0, 0.25]),
                               atol=1e-15)


@pytest.mark.parametrize("chain", [2, 5])
def test_se3_chain_equals_sequential_application(chain):
    """Composing T0..T_{c-1} then applying equals applying T_{c-1} first, then
    ..., T0 last, one transform at a time."""
    b, npts = 3, 20
    T = W.se3_transforms(b * chain, 140 + chain).astype(np.float64)
    Tm = _mats(T, b * chain, 4, 4).reshape(b, chain, 4, 4)
    Tm[:, :, 3, :] = 777.0                  # the bottom row must never be read
    P = W.gaussian(b * 3 * npts, 141).astype(np.float64)
    Q = oracle.se3_apply(chain, _cm(Tm.reshape(-1, 4, 4)), npts, P, b)
    cur = P
    for c in reversed(range(chain)):
        cur = oracle.se3_apply(1, _cm(Tm[:, c]), npts, cur, b)
    np.testing.assert_allclose(Q, cur, atol=1e-12)


# ------------------------------------------------------------- cost model
DIN, H, DOUT = 8, 64, 12


def _mlp_case(rows=7, seed=150):
    g = W.rng(seed)
    w = g.standard_normal(oracle.mlp_nparams(DIN, H, DOUT)) * 0.3
    X = g.standard_normal((rows, DIN))
    T = g.standard_normal((rows, DOUT))
    M = (g.random((rows, DOUT)) > 0.3).astype(np.float64)
    return w, X, T, M


def test_mlp_param_count():
    assert oracle.mlp_nparams(8, 64, 12) == 5516


def test_mlp_closed_form_bias_only():
    w = np.zeros(oracle.mlp_nparams(DIN, H, DOUT))
    w[-DOUT:] = np.arange(DOUT) * 0.5          # only b3 non-zero: y = b3
    X = W.rng(151).standard_normal((3, DIN))
    Y = oracle.mlp_fwd(DIN, H, DOUT, w, X)
    np.testing.assert_array_equal(Y, np.broadcast_to(w[-DOUT:], (3, DOUT)))
    T = np.zeros((3, DOUT))
    M = np.ones((3, DOUT))
    loss, g = oracle.mlp_loss_grad(DIN, H, DOUT, w, X, T, M)
    assert loss == pytest.approx(np.sum(w[-DOUT:] ** 2) * 3 / (3 * DOUT))
    np.testing.assert_allclose(g[-DOUT:], 2 * 3 * w[-DOUT:] / (3 * DOUT))
    assert np.all(g[:-DOUT] == 0)


def test_mlp_forward_matches_numpy_layers():
    w, X, _, _ = _mlp_case()
    o = [0, H * DIN, H * DIN + H, H * DIN + H + H * H, H * DIN + 2 * H + H * H,
         H * DIN + 2 * H + H * H + DOUT * H]
    W1 = w[o[0]:o[1]].reshape(H, DIN); b1 = w[o[1]:o[2]]
    W2 = w[o[2]:o[3]].reshape(H, H); b2 = w[o[3]:o[4]]
    W3 = w[o[4]:o[5]].reshape(DOUT, H); b3 = w[o[5]:]
    ref = np.maximum(np.maximum(X @ W1.T + b1, 0) @ W2.T + b2, 0) @ W3.T + b3
    np.testing.assert_allclose(oracle.mlp_fwd(DIN, H, DOUT, w, X), ref, rtol=1e-12, atol=1e-12)


def test_mlp_gradient_vs_central_differences():
    w, X, T, M = _mlp_case()
    _, g = oracle.mlp_loss_grad(DIN, H, DOUT, w, X, T, M)
    idx = W.rng(152).choice(w.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        wp = w.copy(); wp[i] += h
        wm = w.copy(); wm[i] -= h
        lp, _ = oracle.mlp_loss_grad(DIN, H, DOUT, wp, X, T, M)
        lm, _ = oracle.mlp_loss_grad(DIN, H, DOUT, wm, X, T, M)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_closed_form_and_training_decreases():
    w = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 0.0])
    m = np.zeros(3); v = np.zeros(3)
    oracle.adam_step(w, g, m, v, 1, lr=0.1)
    # step 1: m_hat = g, v_hat = g^2 -> update = lr * g / (|g| + eps)
    np.testing.assert_allclose(w, [1.0 - 0.1 * 0.5 / (0.5 + 1e-8),
                                   -2.0 + 0.1 * 4.0 / (4.0 + 1e-8), 3.0])
    wv, X, T, M = _mlp_case(rows=64, seed=153)
    mm = np.zeros_like(wv); vv = np.zeros_like(wv)
    l0, _ = oracle.mlp_loss_grad(DIN, H, DOUT, wv, X, T, M)
    for t in range(1, 101):
        _, gr = oracle.mlp_loss_grad(DIN, H, DOUT, wv, X, T, M)
        oracle.adam_step(wv, gr, mm, vv, t, lr=1e-2)
    l1, _ = oracle.mlp_loss_grad(DIN, H, DOUT, wv, X, T, M)
    assert l1 < 0.5 * l0


# ------------------------------------------------------- gemm with op()
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_ex_matches_numpy_with_transposes_and_scaling(ta, tb):
    rng = np.random.default_rng(40 + 2 * ta + tb)
    m, n, k, batch = 5, 7, 4, 6
    A = rng.standard_normal((batch, k, m) if ta else (batch, m, k))
    B = rng.standard_normal((batch, n, k) if tb else (batch, k, n))
    C = rng.standard_normal((batch, m, n))
    lda, ldb, ldc = A.shape[1] + 2, B.shape[1] + 1, m + 3

    def pad(X, ld):
        out = np.zeros((X.shape[0], X.shape[2], ld))
        out[:, :, :X.shape[1]] = X.transpose(0, 2, 1)
        return out.reshape(-1), ld * X.shape[2]
    a, sA = pad(A, lda)
    b, sB = pad(B, ldb)
    c, sC = pad(C, ldc)
    got = oracle.gemm_ex(ta, tb, m, n, k, 1.5, a, lda, sA, b, ldb, sB, -0.5, c, ldc, sC, batch)
    opA = A.transpose(0, 2, 1) if ta else A
    opB = B.transpose(0, 2, 1) if tb else B
    want = 1.5 * opA @ opB - 0.5 * C
    got = got.reshape(batch, n, ldc).transpose(0, 2, 1)[:, :m]
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # beta == 0 never reads C (NaN there stays out of the result)
    nanc = np.full_like(c, np.nan)
    got0 = oracle.gemm_ex(ta, tb, m, n, k, 2.0, a, lda, sA, b, ldb, sB, 0.0, nanc, ldc, sC, batch)
    got0 = got0.reshape(batch, n, ldc).transpose(0, 2, 1)[:, :m]
    assert np.abs(got0 - 2.0 * opA @ opB).max() <= 1e-12 * np.abs(opA @ opB).max()


def test_gemm_ex_integer_exact():
    rng = np.random.default_rng(44)
    m = n = k = 9
    A = rng.integers(-4, 5, size=(3, m, k)).astype(np.float64)
    B = rng.integers(-4, 5, size=(3, k, n)).astype(np.float64)
    got = oracle.gemm_ex(1, 0, m, n, k, 1.0, _cm(A.transpose(0, 2, 1)), k, m * k, _cm(B), k, k * n, 0.0, None, m,
                         m * n, 3)
    assert np.array_equal(_mats(got, 3, m, n), A @ B)


# ------------------------------------------------------- LQR gain
def _riccati_case(nx, nu, batch, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(nx) + 0.1 * rng.standard_normal((batch, nx, nx))
    B = rng.standard_normal((batch, nx, nu))
    Mp = rng.standard_normal((batch, nx, nx))
    P = Mp @ Mp.transpose(0, 2, 1) + nx * np.eye(nx)
    Mr = rng.standard_normal((batch, nu, nu))
    R = Mr @ Mr.transpose(0, 2, 1) + nu * np.eye(nu)
    return A, B, P, R


@pytest.mark.parametrize("nx,nu", [(1, 1), (4, 1), (6, 3), (12, 4), (14, 7)])
def test_riccati_gain_matches_linear_solve(nx, nu):
    batch = 7
    A, B, P, R = _riccati_case(nx, nu, batch, 50 + nx)
    K, info = oracle.riccati_gain(nx, nu, _cm(A), _cm(B), _cm(P), _cm(R), batch)
    Bt = B.transpose(0, 2, 1)
    want = np.linalg.solve(R + Bt @ P @ B, Bt @ P @ A)
    assert (info == 0).all()
    assert np.abs(_mats(K, batch, nu, nx) - want).max() <= 1e-10 * np.abs(want).max()


def test_riccati_gain_scalar_closed_form():
    a, b, p, r = 1.25, -0.75, 3.0, 0.5
    K, info = oracle.riccati_gain(1, 1, [a], [b], [p], [r], 1)
    assert info[0] == 0 and K[0] == pytest.approx(b * p * a / (r + b * b * p), rel=1e-15)


def test_riccati_gain_dyadic_exact():
    # B = P = I, R = 3 I (nu = nx): S = 4 I, L = 2 I, K = A / 4 exactly
    nx, batch = 5, 4
    A = np.random.default_rng(51).integers(-8, 9, size=(batch, nx, nx)).astype(np.float64)
    I = np.broadcast_to(np.eye(nx), (batch, nx, nx))
    K, info = oracle.riccati_gain(nx, nx, _cm(A), _cm(I), _cm(I), _cm(3 * I), batch)
    assert (info == 0).all() and np.array_equal(_mats(K, batch, nx, nx), A / 4)


def test_riccati_gain_satisfies_the_discrete_riccati_equation():
    # P from SciPy's DARE solver; the oracle's K must close the Riccati
    # recursion P = Q + A^T P A - A^T P B K (a transposed operand fails it)
    rng = np.random.default_rng(52)
    nx, nu = 6, 2
    A = np.eye(nx) + 0.2 * rng.standard_normal((nx, nx))
    B = rng.standard_normal((nx, nu))
    Q = np.eye(nx)
    R = np.array([[2.0, 0.3], [0.3, 1.0]])
    P = sla.solve_discrete_are(A, B, Q, R)
    K, info = oracle.riccati_gain(nx, nu, _cm(A[None]), _cm(B[None]), _cm(P[None]), _cm(R[None]), 1)
    K = _mats(K, 1, nu, nx)[0]
    assert info[0] == 0
    resid = Q + A.T @ P @ A - A.T @ P @ B @ K - P
    assert np.abs(resid).max() <= 1e-9 * np.abs(P).max()


def test_riccati_gain_reports_indefinite_s():
    # B = 0 leaves S = R; an R whose second pivot is negative gives info = 2
    nx, nu = 3, 2
    A = np.eye(nx)[None]
    B = np.zeros((1, nx, nu))
    P = np.eye(nx)[None]
    R = np.array([[[1.0, 2.0], [2.0, 1.0]]])
    _, info = oracle.riccati_gain(nx, nu, _cm(A), _cm(B), _cm(P), _cm(R), 1)
    assert info[0] == 2


# ------------------------------------------------- robotics operations
def _unit_quats(batch, seed):
    q = np.random.default_rng(seed).standard_normal((batch, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _wxyz_to_scipy(q):
    from scipy.spatial.transform import Rotation
    return Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], axis=1))


@pytest.mark.parametrize("scale", [1.0, 1e-3, 1e-9, 0.0])
def test_quat_retract_against_scipy_rotations(scale):
    from scipy.spatial.transform import Rotation
    batch = 40
    q = _unit_quats(batch, 100)
    d = scale * np.random.default_rng(101).standard_normal((batch, 3))
    out = oracle.quat_retract(q.reshape(-1), d.reshape(-1), batch).reshape(batch, 4)
    want = (_wxyz_to_scipy(q) * Rotation.from_rotvec(d)).as_matrix()
    assert np.abs(_wxyz_to_scipy(out).as_matrix() - want).max() <= 1e-13
    assert np.abs(np.linalg.norm(out, axis=1) - 1.0).max() <= 1e-14
    if scale == 0.0:
        assert np.array_equal(out, q)


@pytest.mark.parametrize("scale", [1.0, 1e-6, 0.0])
def test_quat_error_inverts_retract_and_matches_scipy(scale):
    batch = 40
    q1 = _unit_quats(batch, 102)
    d = scale * np.random.default_rng(103).uniform(-1, 1, (batch, 3))   # |d| < pi: Log is unique
    q2 = oracle.quat_retract(q1.reshape(-1), d.reshape(-1), batch).reshape(batch, 4)
    q2[::2] *= -1.0                                                     # the double cover
    err = oracle.quat_error(q1.reshape(-1), q2.reshape(-1), batch).reshape(batch, 3)
    assert np.abs(err - d).max() <= 1e-12 * scale + 1e-15          # roundoff of the unit products
    rel = (_wxyz_to_scipy(q1).inv() * _wxyz_to_scipy(q2)).as_rotvec()
    assert np.abs(err - rel).max() <= 1e-12


@pytest.mark.parametrize("scale", [1.0, 1e-3, 1e-8, 0.0])
def test_se3_retract_against_matrix_exponential(scale):
    batch = 20
    rng = np.random.default_rng(104)
    T = np.zeros((batch, 4, 4))
    T[:, :3, :3] = _wxyz_to_scipy(_unit_quats(batch, 105)).as_matrix()
    T[:, :3, 3] = rng.standard_normal((batch, 3))
    T[:, 3, 3] = 1.0
    xi = scale * rng.standard_normal((batch, 6))
    out = oracle.se3_retract(_cm(T), xi.reshape(-1), batch)
    for b in range(batch):
        rho, phi = xi[b, :3], xi[b, 3:]
        Xi = np.zeros((4, 4))
        Xi[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
        Xi[:3, 3] = rho
        want = T[b] @ sla.expm(Xi)
        got = _mats(out[b * 16:(b + 1) * 16], 1, 4, 4)[0]
        assert np.abs(got - want).max() <= 1e-13, (b, scale)


def test_motion_cross_against_the_6x6_cross_matrix():
    batch = 30
    rng = np.random.default_rng(106)
    v, m = rng.standard_normal((batch, 6)), rng.standard_normal((batch, 6))
    out = oracle.motion_cross(v.reshape(-1), m.reshape(-1), batch).reshape(batch, 6)

    def sk(p):
        return np.array([[0, -p[2], p[1]], [p[2], 0, -p[0]], [-p[1], p[0], 0]])
    for b in range(batch):
        vl, w = v[b, :3], v[b, 3:]
        X = np.zeros((6, 6))          # motion cross matrix for (linear, angular) ordering
        X[:3, :3] = sk(w)
        X[:3, 3:] = sk(vl)
        X[3:, 3:] = sk(w)
        assert np.abs(out[b] - X @ m[b]).max() <= 1e-14
    vv = oracle.motion_cross(v.reshape(-1), v.reshape(-1), batch)
    assert np.abs(vv).max() <= 1e-14                         # v x v = 0


def test_eig3_against_numpy_eigh():
    batch = 60
    rng = np.random.default_rng(107)
    A = rng.standard_normal((batch, 3, 3))
    A = A + A.transpose(0, 2, 1)
    A[0] = np.diag([3.0, -1.0, 2.0])                          # already diagonal
    A[1] = 2.0 * np.eye(3)                                    # triple eigenvalue
    w, V = oracle.eig3(_cm(A), batch)
    w, V = w.reshape(batch, 3), _mats(V, batch, 3, 3)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() <= 1e-13
    assert np.abs(A @ V - V * w[:, None, :]).max() <= 1e-13
    assert np.abs(V.transpose(0, 2, 1) @ V - np.eye(3)).max() <= 1e-13
    big = np.argmax(np.abs(V), axis=1)
    assert (np.take_along_axis(V, big[:, None, :], axis=1) > 0).all()


def test_svd3_against_numpy_and_closest_rotation_against_polar():
    batch = 60
    rng = np.random.default_rng(108)
    M = rng.standard_normal((batch, 3, 3))
    M[0] = np.diag([1.0, 2.0, 0.0])                            # rank deficient
    U, s, V = oracle.svd3(_cm(M), batch)
    U, s, V = _mats(U, batch, 3, 3), s.reshape(batch, 3), _mats(V, batch, 3, 3)
    assert np.abs(s - np.linalg.svd(M, compute_uv=False)).max() <= 1e-12
    assert np.abs(U * s[:, None, :] @ V.transpose(0, 2, 1) - M).max() <= 1e-12
    assert np.abs(U.transpose(0, 2, 1) @ U - np.eye(3)).max() <= 1e-12
    R = _mats(oracle.closest_rotation(_cm(M), batch), batch, 3, 3)
    assert np.abs(R.transpose(0, 2, 1) @ R - np.eye(3)).max() <= 1e-12
    assert np.abs(np.linalg.det(R) - 1.0).max() <= 1e-12
    pos = np.linalg.det(M) > 0
    for b in np.nonzero(pos)[0]:
        Up, _ = sla.polar(M[b])                                # orthogonal polar factor = closest rotation
        assert np.abs(R[b] - Up).max() <= 1e-11
    # the closest rotation to a rotation is itself
    Q = _wxyz_to_scipy(_unit_quats(5, 109)).as_matrix()
    assert np.abs(_mats(oracle.closest_rotation(_cm(Q), 5), 5, 3, 3) - Q).max() <= 1e-13


def test_argmax_and_softmax_against_numpy():
    from scipy.special import softmax as sp_softmax
    batch, n = 50, 16
    x = np.random.default_rng(110).standard_normal((batch, n))
    x[3, [2, 9]] = 7.0                                          # tie: the first index wins
    assert np.array_equal(oracle.argmax(n, x.reshape(-1), batch), np.argmax(x, axis=1))
    assert oracle.argmax(n, x.reshape(-1), batch)[3] == 2
    y = oracle.softmax(n, x.reshape(-1), batch).reshape(batch, n)
    assert np.abs(y - sp_softmax(x, axis=1)).max() <= 1e-15
    big = oracle.softmax(n, (x + 1000.0).reshape(-1), batch).reshape(batch, n)  # shift invariance, no overflow
    assert np.abs(big - y).max() <= 1e-12                       # x + 1000 rounds at ~1e-13


# ------------------------------------------- BLAS-1/2 and block-tridiagonal
def test_dot_and_gemv_against_numpy():
    rng = np.random.default_rng(120)
    batch, n = 9, 37
    x, y = rng.standard_normal((batch, n + 2)), rng.standard_normal((batch, n + 5))
    got = oracle.dot(n, x.reshape(-1), y.reshape(-1), batch, sx=n + 2, sy=n + 5)
    assert np.abs(got - np.einsum("bi,bi->b", x[:, :n], y[:, :n])).max() <= 1e-13
    assert oracle.dot(3, [1.0, 2.0, 3.0], [4.0, -5.0, 6.0], 1)[0] == 12.0
    m, k = 6, 5
    A = rng.standard_normal((batch, m, k))
    lda = m + 1
    a, sA = np.zeros((batch, k, lda)), k * lda
    a[:, :, :m] = A.transpose(0, 2, 1)
    for trans in (0, 1):
        xin = rng.standard_normal((batch, m if trans else k))
        yin = rng.standard_normal((batch, k if trans else m))
        out = oracle.gemv(trans, m, k, 2.0, a.reshape(-1), lda, sA, xin.reshape(-1), xin.shape[1], -1.0,
                          yin.reshape(-1), yin.shape[1], batch).reshape(batch, -1)
        opA = A.transpose(0, 2, 1) if trans else A
        want = 2.0 * np.einsum("bij,bj->bi", opA, xin) - yin
        assert np.abs(out - want).max() <= 1e-13


def _btd_case(nb, N, batch, seed, shift=None):
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((batch, N, nb, nb))
    D = D @ D.transpose(0, 1, 3, 2) + (2.0 * nb + 2.0 if shift is None else shift) * np.eye(nb)
    O = rng.standard_normal((batch, max(N - 1, 1), nb, nb))[:, :max(N - 1, 0)]
    return D, O


def _btd_dense(D, O):
    batch, N, nb = D.shape[0], D.shape[1], D.shape[2]
    T = np.zeros((batch, N * nb, N * nb))
    for i in range(N):
        T[:, i * nb:(i + 1) * nb, i * nb:(i + 1) * nb] = D[:, i]
        if i + 1 < N:
            T[:, (i + 1) * nb:(i + 2) * nb, i * nb:(i + 1) * nb] = O[:, i]
            T[:, i * nb:(i + 1) * nb, (i + 1) * nb:(i + 2) * nb] = O[:, i].transpose(0, 2, 1)
    return T


def _btd_flat(X):
    return np.ascontiguousarray(X.transpose(0, 1, 3, 2)).reshape(-1)     # column-major blocks


@pytest.mark.parametrize("nb,N", [(1, 1), (1, 7), (3, 5), (6, 10), (12, 4)])
def test_btd_matvec_and_solve_against_banded_cholesky(nb, N):
    batch = 5
    D, O = _btd_case(nb, N, batch, 130 + nb + N)
    rng = np.random.default_rng(131)
    x = rng.standard_normal((batch, N * nb))
    y = oracle.btd_matvec(nb, N, _btd_flat(D), _btd_flat(O), x.reshape(-1), batch).reshape(batch, -1)
    T = _btd_dense(D, O)
    assert np.abs(y - np.einsum("bij,bj->bi", T, x)).max() <= 1e-12 * np.abs(y).max()
    b = rng.standard_normal((batch, N * nb))
    X, info = oracle.btd_posv(nb, N, _btd_flat(D), _btd_flat(O), b.reshape(-1), batch)
    assert (info == 0).all()
    X = X.reshape(batch, -1)
    for k in range(batch):
        # SciPy's banded Cholesky (lower form, bandwidth 2nb-1): an independent solver
        m, u = N * nb, 2 * nb - 1
        ab = np.zeros((u + 1, m))
        for d in range(u + 1):
            ab[d, :m - d] = np.diagonal(T[k], -d)
        cb = sla.cholesky_banded(ab, lower=True)
        want = sla.cho_solve_banded((cb, True), b[k])
        assert np.abs(X[k] - want).max() <= 1e-11 * np.abs(want).max()


def test_btd_scalar_tridiagonal_closed_form_and_info():
    # nb = 1: the 1-D Laplacian tridiag(-1, 2, -1) of order 4 with b = (1,0,0,1): x = (1,1,1,1)
    D = np.full((1, 4, 1, 1), 2.0)
    O = np.full((1, 3, 1, 1), -1.0)
    X, info = oracle.btd_posv(1, 4, _btd_flat(D), _btd_flat(O), [1.0, 0.0, 0.0, 1.0], 1)
    assert info[0] == 0 and np.abs(X - 1.0).max() <= 1e-15
    # an indefinite second diagonal block: the dense factor fails in its first column (global 3)
    D, O = _btd_case(2, 3, 1, 132)
    D[0, 1] = -np.eye(2)
    O[:] = 0.0
    _, info = oracle.btd_posv(2, 3, _btd_flat(D), _btd_flat(O), np.zeros(6), 1)
    assert info[0] == 3


# ------------------------------------------------ block-Jacobi PCG (iterative)
def _btd_spd(nb, N, batch, seed):
    """An SPD block-tridiagonal case (off-diagonal blocks halved; positive
    definiteness checked with numpy.linalg.eigvalsh)."""
    D, O = _btd_case(nb, N, batch, seed)
    O = 0.5 * O
    assert (np.linalg.eigvalsh(_btd_dense(D, O)) > 0).all()
    return D, O


def _blockdiag_inverse(D):
    """Dense inverse of blockdiag(D_0..D_{N-1}) of one problem (numpy.linalg.inv per block)."""
    N, nb = D.shape[0], D.shape[1]
    M = np.zeros((N * nb, N * nb))
    for i in range(N):
        M[i * nb:(i + 1) * nb, i * nb:(i + 1) * nb] = np.linalg.inv(D[i])
    return M


@pytest.mark.parametrize("nb,N", [(1, 9), (3, 5), (6, 4)])
def test_btd_pcg_iterates_match_scipy_cg(nb, N):
    """Each PCG iterate equals SciPy's preconditioned CG iterate (same x0,
    preconditioner blockdiag(D)^-1, no tolerance stop) for k = 1..6."""
    from scipy.sparse.linalg import cg
    batch = 3
    D, O = _btd_spd(nb, N, batch, 140 + nb)
    T = _btd_dense(D, O)
    rng = np.random.default_rng(141)
    b = rng.standard_normal((batch, N * nb))
    x0 = rng.standard_normal((batch, N * nb))
    for k in range(1, 7):
        X, done = oracle.btd_pcg(nb, N, _btd_flat(D), _btd_flat(O), b.reshape(-1), x0.reshape(-1), k, 0.0, batch)
        X = X.reshape(batch, -1)
        assert (done == k).all()
        for p in range(batch):
            its = []
            cg(T[p], b[p], x0=x0[p].copy(), rtol=0.0, atol=0.0, maxiter=k, M=_blockdiag_inverse(D[p]),
               callback=lambda xk: its.append(xk.copy()))
            assert len(its) == k
            assert np.abs(X[p] - its[-1]).max() <= 1e-10 * np.abs(its[-1]).max(), (k, p)


def test_btd_pcg_converges_to_the_direct_solve_and_lowers_the_energy_error():
    """In exact arithmetic CG ends within N*nb steps; the FP64 iterate then
    matches SciPy's banded Cholesky solve, and the T-norm of the error never
    grows from one iterate to the next (CG minimises it over the Krylov space)."""
    nb, N, batch = 4, 6, 2
    D, O = _btd_spd(nb, N, batch, 150)
    T = _btd_dense(D, O)
    b = np.random.default_rng(151).standard_normal((batch, N * nb))
    x0 = np.zeros_like(b)
    want = np.linalg.solve(T, b[..., None])[..., 0]
    prev = None
    for k in range(0, N * nb + 1):
        X, _ = oracle.btd_pcg(nb, N, _btd_flat(D), _btd_flat(O), b.reshape(-1), x0.reshape(-1), k, 0.0, batch)
        e = X.reshape(batch, -1) - want
        energy = np.einsum("bi,bij,bj->b", e, T, e)
        if prev is not None:
            assert (energy <= prev * (1 + 1e-9) + 1e-24).all(), k
        prev = energy
    assert np.abs(e).max() <= 1e-8 * np.abs(want).max()


def test_btd_pcg_exact_preconditioner_and_failure():
    """A single block (or zero off-diagonal blocks) makes the preconditioner
    T itself: one iteration solves the system and the tolerance stops the
    loop there; a non-SPD diagonal block gives iters_done = -1 and leaves x."""
    for nb, N in ((5, 1), (3, 4)):
        D, O = _btd_case(nb, N, 2, 160 + N)
        O[:] = 0.0
        b = np.random.default_rng(161).standard_normal((2, N * nb))
        X, done = oracle.btd_pcg(nb, N, _btd_flat(D), _btd_flat(O), b.reshape(-1), np.zeros(2 * N * nb), 10, 1e-8, 2)
        assert (done == 1).all()
        want = np.linalg.solve(_btd_dense(D, O), b[..., None])[..., 0]
        assert np.abs(X.reshape(2, -1) - want).max() <= 1e-12 * np.abs(want).max()
    D, O = _btd_case(2, 3, 1, 162)
    D[0, 2] = -np.eye(2)
    x0 = np.arange(6.0)
    X, done = oracle.btd_pcg(2, 3, _btd_flat(D), _btd_flat(O), np.ones(6), x0, 5, 0.0, 1)
    assert done[0] == -1 and np.array_equal(X, x0)
