"""Parity of the CUDA path against the FP64 oracle, through the C ABI.

Every op runs at every feasible placement (scope x pack) on sizes that span
several tiles with ragged tails.  Bars:
  - integer / index results (pivots, info) bit-exact;
  - exact-arithmetic inputs (integer / dyadic constructions) bit-exact;
  - FP32 results: solves within 1e-4 normwise backward error (the stated
    relative-residual bar) and, problem by problem, within 1e-4 of the
    oracle scaled by that problem's largest entry (the inputs are well
    conditioned, kappa < 1e2); LU factors also within the rounding-error
    bound of the factorization itself, entry by entry;
  - GEMM elementwise within the classical bound k * 2^-23 * (|A||B|)_ij.
"""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W
from tests.helpers import (U32, backward_error, dev, host, lower_mask, opts_for, per_problem_rel, placements, sync,
                           to_dev, zeros_i32)

pytestmark = pytest.mark.gpu

NS = [1, 2, 3, 5, 6, 7, 12, 14, 16, 24, 31, 32, 33, 64]
BATCH = 300  # > 256 (largest thread-scope CTA) and not a multiple of 32


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


def mats(flat, batch, r, c):
    return W.from_colmajor(flat, batch, r, c)


# ------------------------------------------------------------------- gemm
@pytest.mark.parametrize("n", NS)
def test_gemm_all_placements(n):
    batch = BATCH
    A = W.gaussian(batch * n * n, 1 + n)
    B = W.gaussian(batch * n * n, 2 + n)
    ref = oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch)
    bound = n * 2 * U32 * (np.abs(mats(A, batch, n, n)) @ np.abs(mats(B, batch, n, n))) + 1e-30
    dA, dB = to_dev(A), to_dev(B)
    for scope, pack in placements(g.GLASS_OP_GEMM, n, n):
        dC = to_dev(np.full(batch * n * n, np.nan, np.float32))
        g.check(g.glass_batched_gemm(n, n, n, dA, n, n * n, dB, n, n * n, dC, n, n * n, batch,
                                     opts_for(scope, pack)), f"gemm {n} {scope} {pack}")
        sync()
        err = np.abs(mats(host(dC).astype(np.float64) - ref, batch, n, n)) / bound
        assert err.max() <= 1.0, (n, scope, pack, err.max())


@pytest.mark.parametrize("m,n,k", [(5, 7, 3), (16, 8, 33), (64, 1, 64), (1, 64, 17)])
def test_gemm_rectangular_and_strided(m, n, k):
    batch = 70
    lda, ldb, ldc = m + 3, k + 1, m + 2
    sA, sB, sC = lda * k + 5, ldb * n, ldc * n + 7
    A = W.gaussian(batch * sA, 11)
    B = W.gaussian(batch * sB, 12)
    ref = oracle.gemm(m, n, k, A.astype(np.float64), B.astype(np.float64), batch, lda=lda, ldb=ldb, ldc=ldc,
                      sA=sA, sB=sB, sC=sC)
    for scope, pack in [(1, 1), (1, 4), (2, 1), (2, 2)] + ([(0, 1), (0, 8)] if max(m, n, k) <= 8 else []):
        if not g.glass_placement_feasible(g.GLASS_OP_GEMM, max(m, n, k), max(m, n, k), scope, pack):
            continue
        dC = to_dev(np.zeros(batch * sC, np.float32))
        s = g.glass_batched_gemm(m, n, k, to_dev(A), lda, sA, to_dev(B), ldb, sB, dC, ldc, sC, batch,
                                 opts_for(scope, pack))
        g.check(s, "gemm rect")
        sync()
        C = host(dC).astype(np.float64)
        for b in (0, 1, batch - 1):
            got = C[b * sC:b * sC + ldc * n].reshape(n, ldc).T[:m]
            want = ref[b * sC:b * sC + ldc * n].reshape(n, ldc).T[:m]
            np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("n", [3, 8, 16, 32, 64])
def test_gemm_integer_bit_exact(n):
    batch = 65
    A = W.colmajor(W.int_matrix(n, n, batch, 200 + n))
    B = W.colmajor(W.int_matrix(n, n, batch, 300 + n))
    ref = oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch)
    for scope, pack in placements(g.GLASS_OP_GEMM, n, n):
        dC = to_dev(np.zeros(batch * n * n, np.float32))
        g.check(g.glass_batched_gemm(n, n, n, to_dev(A), n, n * n, to_dev(B), n, n * n, dC, n, n * n, batch,
                                     opts_for(scope, pack)))
        sync()
        assert np.array_equal(host(dC).astype(np.float64), ref), (n, scope, pack)


# --------------------------------------------------------------- cholesky
def _spd_case(n, batch, seed):
    A = W.spd(n, batch, seed)
    return A


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("nrhs", [1, 4])
def test_posv_all_placements(n, nrhs):
    batch = BATCH
    A = _spd_case(n, batch, 400 + n)
    B = W.gaussian(batch * n * nrhs, 401 + n)
    L_ref, X_ref, info_ref = oracle.posv(n, nrhs, A.astype(np.float64), B.astype(np.float64), batch)
    assert (info_ref == 0).all()
    Am = mats(A, batch, n, n).astype(np.float64)
    Bm = mats(B, batch, n, nrhs).astype(np.float64)
    for scope, pack in placements(g.GLASS_OP_POSV, n, nrhs):
        dA, dB, info = to_dev(A), to_dev(B), zeros_i32(batch)
        g.check(g.glass_batched_posv(n, nrhs, dA, n, n * n, dB, n, n * nrhs, info, batch,
                                     opts_for(scope, pack)), f"posv {n} {scope} {pack}")
        sync()
        assert (host(info)[:batch] == 0).all()
        X = host(dB).astype(np.float64)
        L = host(dA).astype(np.float64)
        tag = (n, nrhs, scope, pack)
        assert per_problem_rel(X, X_ref, batch) <= 1e-4, tag
        assert per_problem_rel(L, L_ref, batch, lower_mask(n)) <= 1e-4, tag
        # upper triangle left as it was
        up = np.triu_indices(n, 1)
        assert np.array_equal(mats(L, batch, n, n)[:, up[0], up[1]], Am[:, up[0], up[1]]), tag
        assert backward_error(Am, mats(X, batch, n, nrhs), Bm).max() <= 1e-4, tag


@pytest.mark.parametrize("n", [2, 6, 12, 16, 24, 40, 64])
def test_potrf_potrs_integer_bit_exact(n):
    batch = 70
    A, L0 = W.int_cholesky_factor(n, batch, 500 + n)
    X0 = W.int_matrix(n, 2, batch, 501 + n, -3, 3)
    B = A @ X0
    Acm, Bcm = W.colmajor(A), W.colmajor(B)
    for scope, pack in placements(g.GLASS_OP_POSV, n, 2):
        dA, dB, info = to_dev(Acm), to_dev(Bcm), zeros_i32(batch)
        g.check(g.glass_batched_potrf(n, dA, n, n * n, info, batch, opts_for(scope, pack)))
        g.check(g.glass_batched_potrs(n, 2, dA, n, n * n, dB, n, 2 * n, batch, opts_for(scope, pack)))
        sync()
        assert (host(info)[:batch] == 0).all()
        assert np.array_equal(np.tril(mats(host(dA), batch, n, n)), L0), (n, scope, pack)
        assert np.array_equal(mats(host(dB), batch, n, 2), X0), (n, scope, pack)


@pytest.mark.parametrize("n", [1, 5, 8, 33])
def test_potrf_reports_first_failing_column(n):
    batch = 40
    A, L0 = W.int_cholesky_factor(n, batch, 600 + n)
    rng = W.rng(601)
    fail = rng.integers(0, n, size=batch)
    bad = rng.random(batch) < 0.5
    for b in range(batch):
        if bad[b]:
            j = fail[b]
            A[b, j, j] -= L0[b, j, j] ** 2 + 1.0
    want = np.where(bad, fail + 1, 0)
    for scope, pack in placements(g.GLASS_OP_POTRF, n, 1):
        dA, info = to_dev(W.colmajor(A)), zeros_i32(batch)
        g.check(g.glass_batched_potrf(n, dA, n, n * n, info, batch, opts_for(scope, pack)))
        sync()
        assert np.array_equal(host(info)[:batch], want), (n, scope, pack)


@pytest.mark.parametrize("n", NS)
def test_trsm_square_rhs_all_placements(n):
    batch = 130
    k = n
    g0 = W.rng(700 + n)
    L = np.tril(g0.standard_normal((batch, n, n))) + 3.0 * np.eye(n)
    Lcm = W.colmajor(L)
    B = W.gaussian(batch * n * k, 701 + n)
    ref = oracle.trsm(n, k, Lcm.astype(np.float64), B.astype(np.float64), batch)
    for scope, pack in placements(g.GLASS_OP_TRSM, n, k):
        dB = to_dev(B)
        g.check(g.glass_batched_trsm(n, k, to_dev(Lcm), n, n * n, dB, n, n * k, batch, opts_for(scope, pack)))
        sync()
        X = host(dB).astype(np.float64)
        assert per_problem_rel(X, ref, batch) <= 1e-4, (n, scope, pack)


@pytest.mark.parametrize("n", [19, 21, 23])
def test_solves_of_orders_17_to_23(n):
    """Orders 17..23 (the column solve's order-24 bucket, staged element by
    element since n is not a multiple of 4): trsm with n right-hand sides at
    every placement against the oracle, and potrf + potrs recovering integer
    solutions bit for bit at every placement."""
    batch = 70
    g0 = W.rng(760 + n)
    L = np.tril(g0.standard_normal((batch, n, n))) + 3.0 * np.eye(n)
    Lcm = W.colmajor(L)
    B = W.gaussian(batch * n * n, 761 + n)
    ref = oracle.trsm(n, n, Lcm.astype(np.float64), B.astype(np.float64), batch)
    for scope, pack in placements(g.GLASS_OP_TRSM, n, n):
        dB = to_dev(B)
        g.check(g.glass_batched_trsm(n, n, to_dev(Lcm), n, n * n, dB, n, n * n, batch, opts_for(scope, pack)))
        sync()
        assert per_problem_rel(host(dB).astype(np.float64), ref, batch) <= 1e-4, (n, scope, pack)
    A, L0 = W.int_cholesky_factor(n, batch, 770 + n)
    X0 = W.int_matrix(n, 6, batch, 771 + n, -3, 3)
    Acm, Bcm = W.colmajor(A), W.colmajor(A @ X0)
    for scope, pack in placements(g.GLASS_OP_POSV, n, 6):
        dA, dB, info = to_dev(Acm), to_dev(Bcm), zeros_i32(batch)
        g.check(g.glass_batched_potrf(n, dA, n, n * n, info, batch, opts_for(scope, pack)))
        g.check(g.glass_batched_potrs(n, 6, dA, n, n * n, dB, n, 6 * n, batch, opts_for(scope, pack)))
        sync()
        assert (host(info)[:batch] == 0).all()
        assert np.array_equal(mats(host(dB), batch, n, 6), X0), (n, scope, pack)


@pytest.mark.parametrize("n", [33, 40, 64])
def test_lu_team_of_two_warps_matches_one_warp_bit_for_bit(n):
    """The block placement of orders 33..64 runs the tensor-core LU with two
    warps per problem; every element goes through the same operations in the
    same order as in the one-warp form, so factors, interchanges and
    solutions agree bit for bit (Gaussian inputs, where pivots are decided
    by FP32 comparisons of every candidate)."""
    batch = 301
    A = W.general(n, batch, 820 + n)
    b = W.gaussian(batch * n, 821 + n)
    out = {}
    for scope in (g.GLASS_SCOPE_WARP, g.GLASS_SCOPE_BLOCK):
        dA, dB = to_dev(A), to_dev(b)
        ipiv, info = zeros_i32(batch * n), zeros_i32(batch)
        g.check(g.glass_batched_getrf_getrs(n, 1, dA, n, n * n, ipiv, dB, n, n, info, batch, opts_for(scope, 1)))
        sync()
        out[scope] = (host(dA), host(ipiv)[:batch * n], host(dB), host(info)[:batch])
    for a, c in zip(out[g.GLASS_SCOPE_WARP], out[g.GLASS_SCOPE_BLOCK]):
        assert np.array_equal(a.view(np.uint32) if a.dtype == np.float32 else a,
                              c.view(np.uint32) if c.dtype == np.float32 else c), n


@pytest.mark.parametrize("n", [4, 17, 64])
def test_trsm_integer_bit_exact(n):
    batch, k = 40, 5
    L = W.int_lower_pow2_diag(n, batch, 800 + n)
    X0 = W.int_matrix(n, k, batch, 801 + n, -3, 3)
    B = W.colmajor(L @ X0)
    Lg = L.copy()
    Lg[:, np.triu_indices(n, 1)[0], np.triu_indices(n, 1)[1]] = np.nan   # upper never read
    for scope, pack in placements(g.GLASS_OP_TRSM, n, k):
        dB = to_dev(B)
        g.check(g.glass_batched_trsm(n, k, to_dev(W.colmajor(Lg)), n, n * n, dB, n, n * k, batch,
                                     opts_for(scope, pack)))
        sync()
        assert np.array_equal(mats(host(dB), batch, n, k), X0), (n, scope, pack)


# --------------------------------------------------------------------- LU
def _perm_from_ipiv(ipiv, n):
    perm = np.arange(n)
    for j in range(n):
        perm[[j, ipiv[j]]] = perm[[ipiv[j], j]]
    return perm


def _separated_general(n, batch, seed, gap=1e-3):
    """N(0,1) matrices kept only where the oracle's pivot choice is separated
    by a relative gap >= `gap` at every step (distinct pivot magnitudes)."""
    out = []
    s = seed
    while len(out) < batch:
        A = W.gaussian(64 * n * n, s).reshape(64, n * n)
        s += 1
        _, _, _, gp = oracle.getrf(n, A.reshape(-1).astype(np.float64), 64)
        out.extend(A[gp >= gap])
    return np.concatenate(out[:batch]).astype(np.float32)


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("nrhs", [1, 2])
def test_getrf_getrs_all_placements(n, nrhs):
    batch = 200
    A = _separated_general(n, batch, 900 + 10 * n)
    B = W.gaussian(batch * n * nrhs, 901 + n)
    LU_ref, piv_ref, X_ref, info_ref = oracle.getrf_getrs(n, nrhs, A.astype(np.float64), B.astype(np.float64),
                                                          batch)
    _, piv32, _, _ = oracle.getrf(n, A, batch, precision="f32")
    assert np.array_equal(piv32, piv_ref)
    for scope, pack in placements(g.GLASS_OP_GETRF_GETRS, n, nrhs):
        dA, dB = to_dev(A), to_dev(B)
        ipiv, info = zeros_i32(batch * n), zeros_i32(batch)
        g.check(g.glass_batched_getrf_getrs(n, nrhs, dA, n, n * n, ipiv, dB, n, nrhs * n, info, batch,
                                            opts_for(scope, pack)), f"lu {n} {scope} {pack}")
        sync()
        tag = (n, scope, pack)
        assert (host(info)[:batch] == 0).all(), tag
        assert np.array_equal(host(ipiv)[:batch * n], piv_ref), tag
        LU = host(dA).astype(np.float64)
        assert per_problem_rel(LU, LU_ref, batch) <= 1e-4, tag
        # the factorization's own rounding-error bound (Higham, Thm. 9.3):
        # |P A - L U| <= gamma |L||U| entry by entry, with gamma = (2n + 16) u
        # covering FP32 accumulation and the 3xTF32 products of the
        # tensor-core updates (each within 12 u of exact)
        Lf = np.tril(mats(LU, batch, n, n), -1) + np.eye(n)
        Uf = np.triu(mats(LU, batch, n, n))
        Am = mats(A, batch, n, n).astype(np.float64)
        PA = np.stack([Am[b][_perm_from_ipiv(piv_ref[b * n:(b + 1) * n], n)] for b in range(batch)])
        assert (np.abs(PA - Lf @ Uf) <= (2 * n + 16) * U32 * (np.abs(Lf) @ np.abs(Uf)) + 1e-30).all(), tag
        X = host(dB).astype(np.float64)
        assert backward_error(Am, mats(X, batch, n, nrhs), mats(B, batch, n, nrhs).astype(np.float64)).max() <= 1e-4, tag


@pytest.mark.parametrize("n", [2, 6, 12, 24, 64])
def test_getrf_dyadic_bit_exact(n):
    batch = 50
    A, perm, L0, U0 = W.dyadic_lu(n, batch, 1000 + n)
    for scope, pack in placements(g.GLASS_OP_GETRF_GETRS, n, 0):
        dA = to_dev(W.colmajor(A))
        ipiv, info = zeros_i32(batch * n), zeros_i32(batch)
        g.check(g.glass_batched_getrf_getrs(n, 0, dA, n, n * n, ipiv, None, n, n, info, batch,
                                            opts_for(scope, pack)))
        sync()
        LU = mats(host(dA), batch, n, n).astype(np.float64)
        pv = host(ipiv)
        for b in range(batch):
            assert np.array_equal(_perm_from_ipiv(pv[b * n:(b + 1) * n], n), perm[b]), (n, scope, pack)
            assert np.array_equal(np.tril(LU[b], -1) + np.eye(n), L0[b]), (n, scope, pack)
            assert np.array_equal(np.triu(LU[b]), U0[b]), (n, scope, pack)


def test_getrf_singular_info_and_diagonal_dominance():
    n, batch = 7, 64
    A = W.general(n, batch, 1100)        # N(0,1) + n I: pivots on the diagonal
    Am = mats(A, batch, n, n).copy()
    Am[::2, :, 3] = 0.0                   # even problems: zero column 3 -> exact zero pivot at step 3
    Acm = W.colmajor(Am)
    _, piv_ref, info_ref, _ = oracle.getrf(n, Acm, batch, precision="f32")
    for scope, pack in placements(g.GLASS_OP_GETRF_GETRS, n, 1):
        ipiv, info = zeros_i32(batch * n), zeros_i32(batch)
        dB = to_dev(W.gaussian(batch * n, 1101))
        g.check(g.glass_batched_getrf_getrs(n, 1, to_dev(Acm), n, n * n, ipiv, dB, n, n, info, batch,
                                            opts_for(scope, pack)))
        sync()
        inf = host(info)[:batch]
        assert (inf[1::2] == 0).all()
        assert (inf[::2] == 4).all()
        odd = np.concatenate([np.arange(b * n, (b + 1) * n) for b in range(1, batch, 2)])
        assert np.array_equal(host(ipiv)[odd], piv_ref[odd])
        assert np.array_equal(host(ipiv)[odd], np.tile(np.arange(n), batch // 2))


# --------------------------------------------------------------- geometry
@pytest.mark.parametrize("chain", [1, 2, 3, 7, 33, 64])
def test_rot3_compose_all_placements(chain):
    batch = 300
    Rs = W.rotations(batch * chain, 1200 + chain)
    ref = oracle.rot3_compose(chain, Rs.astype(np.float64), batch)
    for scope, pack in placements(g.GLASS_OP_ROT3, 3, chain):
        dR = to_dev(np.zeros(batch * 9, np.float32))
        g.check(g.glass_batched_rot3_compose(chain, to_dev(Rs), 9 * chain, dR, 9, batch, opts_for(scope, pack)))
        sync()
        R = host(dR).astype(np.float64)
        # each 3x3 product of unit-scale rotations adds at most ~9u per entry
        # (three-term dot products whose |terms| sum to <= 3), inputs carry u
        assert np.abs(R - ref).max() <= 12 * (chain + 1) * U32, (chain, scope, pack)
        Rm = mats(R, batch, 3, 3)
        assert np.abs(np.transpose(Rm, (0, 2, 1)) @ Rm - np.eye(3)).max() < 1e-4


# npts 200 and 131: 50 and 32 groups of four points, so the warp scope's two
# prefetched groups per lane exist for some lanes only (or for none) and the
# four-group streaming steps meet ragged ends
@pytest.mark.parametrize("chain,npts", [(1, 1024), (3, 1024), (64, 1024), (2, 7), (5, 1), (7, 200), (33, 131),
                                        (64, 517)])
def test_se3_apply_all_placements(chain, npts):
    batch = 97
    T = W.se3_transforms(batch * chain, 1300 + chain)
    P = W.gaussian(batch * 3 * npts, 1301)
    ref = oracle.se3_apply(chain, T.astype(np.float64), npts, P.astype(np.float64), batch)
    for scope, pack in placements(g.GLASS_OP_SE3, 4, chain):
        dQ = to_dev(np.zeros(batch * 3 * npts, np.float32))
        g.check(g.glass_batched_se3_apply(chain, to_dev(T), 16 * chain, npts, to_dev(P), 3 * npts, dQ, 3 * npts,
                                          batch, opts_for(scope, pack)))
        sync()
        Q = host(dQ).astype(np.float64)
        assert per_problem_rel(Q, ref, batch) <= 12 * (chain + 2) * U32, (chain, npts, scope, pack)


def test_se3_apply_unaligned_points_take_the_scalar_path():
    """Point arrays 4 bytes off a 16-byte boundary: no 16-byte streaming, the
    same result."""
    import torch
    chain, npts, batch = 9, 256, 41
    T = W.se3_transforms(batch * chain, 1320)
    P = W.gaussian(batch * 3 * npts, 1321)
    ref = oracle.se3_apply(chain, T.astype(np.float64), npts, P.astype(np.float64), batch)
    bufP = torch.zeros(batch * 3 * npts + 1, device="cuda")
    bufP[1:] = torch.from_numpy(P).cuda()
    for scope, pack in placements(g.GLASS_OP_SE3, 4, chain):
        bufQ = torch.zeros(batch * 3 * npts + 1, device="cuda")
        g.check(g.glass_batched_se3_apply(chain, to_dev(T), 16 * chain, npts, bufP[1:], 3 * npts, bufQ[1:], 3 * npts,
                                          batch, opts_for(scope, pack)))
        sync()
        Q = bufQ[1:].cpu().numpy().astype(np.float64)
        assert per_problem_rel(Q, ref, batch) <= 12 * (chain + 2) * U32, (scope, pack)


# ---------------------------------------------------------------- layouts
@pytest.mark.parametrize("n", [6, 12, 16])
def test_interleaved_layout_posv_and_roundtrip(n):
    batch = 75
    A = _spd_case(n, batch, 1400 + n)
    B = W.gaussian(batch * n, 1401)
    L_ref, X_ref, _ = oracle.posv(n, 1, A.astype(np.float64), B.astype(np.float64), batch)
    groups = (batch + 31) // 32
    dA, dB = to_dev(A), to_dev(B)
    iA = to_dev(np.full(groups * 32 * n * n, -1, np.float32))
    iB = to_dev(np.full(groups * 32 * n, -1, np.float32))
    g.check(g.glass_to_interleaved32(n, n, dA, iA, batch))
    g.check(g.glass_to_interleaved32(n, 1, dB, iB, batch))
    sync()
    ia = host(iA)
    assert ia[((1 * n * n) + 2 * n + 1) * 32 + 5] == A[(32 + 5) * n * n + 2 * n + 1]   # problem 37, (1,2)
    assert ia[-1] == 0.0                                                                   # pad lane
    info = zeros_i32(batch)
    opts = opts_for(g.GLASS_SCOPE_THREAD, 1, layout=g.GLASS_LAYOUT_INTERLEAVED32)
    g.check(g.glass_batched_posv(n, 1, iA, n, n * n, iB, n, n, info, batch, opts))
    oA, oB = to_dev(np.zeros_like(A)), to_dev(np.zeros_like(B))
    g.check(g.glass_from_interleaved32(n, n, iA, oA, batch))
    g.check(g.glass_from_interleaved32(n, 1, iB, oB, batch))
    sync()
    X = host(oB).astype(np.float64)
    assert per_problem_rel(X, X_ref, batch) <= 1e-4
    assert per_problem_rel(host(oA), L_ref, batch, lower_mask(n)) <= 1e-4
