"""Batched dot, GEMV, TRSV and the block-tridiagonal matvec and solve on the
GPU, through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W
from tests.helpers import U32

pytestmark = pytest.mark.gpu

BATCH = 333


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


def _dev(x, dtype=np.float32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64) if t.dtype != torch.int32 else t.cpu().numpy()


def _nan(n):
    import torch
    return torch.full((max(1, n),), float("nan"), device="cuda")


@pytest.mark.parametrize("n,packed", [(1, False), (7, False), (16, False), (33, False), (100, False),
                                      (1000, False), (16, True), (32, True)])
def test_dot_every_placement(n, packed):
    r = W.rng(300 + n)
    sx, sy = (n, n) if packed else (n + 1, n + 3)   # packed: the 16-byte thread-scope path
    x = r.standard_normal(BATCH * sx).astype(np.float32)
    y = r.standard_normal(BATCH * sy).astype(np.float32)
    ref = oracle.dot(n, x.astype(np.float64), y.astype(np.float64), BATCH, sx=sx, sy=sy)
    absd = oracle.dot(n, np.abs(x).astype(np.float64), np.abs(y).astype(np.float64), BATCH, sx=sx, sy=sy)
    for s, p in [(0, 1), (0, 4), (1, 1), (1, 8), (2, 1), (2, 4), (-1, 0)]:
        out = _nan(BATCH)
        g.check(g.glass_batched_dot(n, _dev(x), sx, _dev(y), sy, out, BATCH, g.make_opts(scope=s, pack=p)))
        assert (np.abs(_host(out)[:BATCH] - ref) <= n * U32 * 2 * absd + 1e-30).all(), (n, s, p)


@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("m,n", [(1, 1), (6, 6), (12, 5), (33, 64), (64, 40)])
def test_gemv_every_placement(trans, m, n):
    r = W.rng(310 + m + n + trans)
    lda = m + 2
    A = r.standard_normal(BATCH * lda * n).astype(np.float32)
    xl, yl = (m, n) if trans else (n, m)
    x = r.standard_normal(BATCH * xl).astype(np.float32)
    y0 = r.standard_normal(BATCH * (yl + 1)).astype(np.float32)
    ref = oracle.gemv(trans, m, n, 0.5, A.astype(np.float64), lda, lda * n, x.astype(np.float64), xl, 2.0,
                      y0.astype(np.float64), yl + 1, BATCH)
    absr = oracle.gemv(trans, m, n, 0.5, np.abs(A).astype(np.float64), lda, lda * n, np.abs(x).astype(np.float64),
                       xl, 2.0, np.abs(y0).astype(np.float64), yl + 1, BATCH)
    for s, p in [(0, 1), (0, 2), (1, 1), (1, 4), (-1, 0)]:
        dy = _dev(y0)
        g.check(g.glass_batched_gemv(trans, m, n, 0.5, _dev(A), lda, lda * n, _dev(x), xl, 2.0, dy, yl + 1, BATCH,
                                     g.make_opts(scope=s, pack=p)))
        got = _host(dy)
        assert (np.abs(got - ref) <= (max(m, n) + 2) * 2 * U32 * absr + 1e-30).all(), (trans, m, n, s, p)
        gaps = got.reshape(BATCH, yl + 1)[:, yl]
        assert np.array_equal(gaps, y0.reshape(BATCH, yl + 1)[:, yl].astype(np.float64))


@pytest.mark.parametrize("n", [3, 17, 64])
def test_trsv_integer_exact(n):
    L = W.int_lower_pow2_diag(n, 40, 320 + n)
    X0 = W.int_matrix(n, 1, 40, 321 + n, -3, 3)
    b = W.colmajor(L @ X0)
    dx = _dev(b)
    g.check(g.glass_batched_trsv(n, _dev(W.colmajor(L)), n, n * n, dx, n, 40))
    assert np.array_equal(_host(dx).reshape(40, n), X0.reshape(40, n))


def _btd(nb, N, batch, seed):
    r = W.rng(seed)
    D = r.standard_normal((batch, N, nb, nb))
    D = D @ D.transpose(0, 1, 3, 2) + (2.0 * nb + 2.0) * np.eye(nb)
    O = r.standard_normal((batch, max(N - 1, 0), nb, nb))
    flat = lambda X: np.ascontiguousarray(X.transpose(0, 1, 3, 2)).reshape(-1).astype(np.float32)
    return flat(D), flat(O) if N > 1 else np.zeros(1, np.float32)


@pytest.mark.parametrize("nb,N", [(1, 1), (1, 9), (3, 5), (6, 16), (12, 8), (16, 3), (32, 2), (7, 33)])
def test_btd_matvec_and_posv(nb, N):
    batch = 67
    D, O = _btd(nb, N, batch, 330 + nb + N)
    r = W.rng(331)
    x = r.standard_normal(batch * N * nb).astype(np.float32)
    yref = oracle.btd_matvec(nb, N, D.astype(np.float64), O.astype(np.float64), x.astype(np.float64), batch)
    yabs = oracle.btd_matvec(nb, N, np.abs(D).astype(np.float64), np.abs(O).astype(np.float64),
                             np.abs(x).astype(np.float64), batch)
    for pack in (1, 4):
        y = _nan(batch * N * nb)
        g.check(g.glass_batched_btd_matvec(nb, N, _dev(D), _dev(O), _dev(x), y, batch, g.make_opts(pack=pack)))
        assert (np.abs(_host(y) - yref) <= 3 * nb * 2 * U32 * yabs + 1e-30).all(), (nb, N, pack)
    b = r.standard_normal(batch * N * nb).astype(np.float32)
    Xref, info = oracle.btd_posv(nb, N, D.astype(np.float64), O.astype(np.float64), b.astype(np.float64), batch)
    assert (info == 0).all()
    for pack in (1, 2, 8):
        dD, dO, db = _dev(D), _dev(O), _dev(b)
        dinfo = _dev(np.full(batch, -5, np.int32), np.int32)
        g.check(g.glass_batched_btd_posv(nb, N, dD, dO, db, dinfo, batch, g.make_opts(pack=pack)))
        assert (_host(dinfo) == 0).all()
        X = _host(db)
        assert np.abs(X - Xref).max() <= 1e-4 * np.abs(Xref).max(), (nb, N, pack)
        # the factor in place: T = L L^T blockwise (check the diagonal blocks' recurrence on one problem)
        Lb = _host(dD).reshape(batch, N, nb, nb).transpose(0, 1, 3, 2)
        Wb = _host(dO).reshape(batch, max(N - 1, 0), nb, nb).transpose(0, 1, 3, 2) if N > 1 else None
        Dm = D.astype(np.float64).reshape(batch, N, nb, nb).transpose(0, 1, 3, 2)
        L0 = np.tril(Lb[0, 0])
        assert np.abs(L0 @ L0.T - Dm[0, 0]).max() <= 1e-5 * np.abs(Dm[0, 0]).max()
        if N > 1:
            Om = O.astype(np.float64).reshape(batch, N - 1, nb, nb).transpose(0, 1, 3, 2)
            assert np.abs(Wb[0, 0] @ L0.T - Om[0, 0]).max() <= 1e-5 * max(1.0, np.abs(Om[0, 0]).max())


def test_btd_posv_reports_the_failing_global_column():
    nb, N, batch = 2, 3, 4
    D, O = _btd(nb, N, batch, 340)
    Dm = D.reshape(batch, N, nb, nb)
    Dm[1::2, 1] = -np.eye(2, dtype=np.float32)        # odd problems: block 1 indefinite
    Om = O.reshape(batch, N - 1, nb, nb)
    Om[1::2] = 0.0
    _, info_ref = oracle.btd_posv(nb, N, D.astype(np.float64), O.astype(np.float64), np.zeros(batch * N * nb), batch)
    dinfo = _dev(np.zeros(batch, np.int32), np.int32)
    g.check(g.glass_batched_btd_posv(nb, N, _dev(D), _dev(O), _dev(np.zeros(batch * N * nb)), dinfo, batch))
    assert np.array_equal(_host(dinfo), info_ref) and (info_ref[1::2] == 3).all()


def _btd_spd(nb, N, batch, seed):
    """SPD block-tridiagonal inputs (the off-diagonal blocks of _btd halved)."""
    D, O = _btd(nb, N, batch, seed)
    return D, (0.5 * O).astype(np.float32)


def _pcg(nb, N, D, O, b, x0, iters, tol, batch, pack=0, ws_bytes=None):
    import torch
    dx = _dev(x0)
    done = _dev(np.full(batch, -7, np.int32), np.int32)
    need = g.glass_btd_pcg_workspace(nb, N, batch)
    ws = torch.empty(max(16, need), dtype=torch.uint8, device="cuda")
    st = g.glass_batched_btd_pcg(nb, N, _dev(D), _dev(O), _dev(b), dx, iters, tol, done, ws,
                                 need if ws_bytes is None else ws_bytes, batch, g.make_opts(pack=pack))
    return st, _host(dx), _host(done)


@pytest.mark.parametrize("nb,N", [(1, 1), (1, 9), (3, 5), (6, 16), (12, 8), (16, 3), (32, 2), (7, 33), (12, 32),
                                  (6, 64)])
def test_btd_pcg_iterates_match_the_oracle(nb, N):
    """After k = 1, 2 and 5 iterations (tol = 0: exactly k) every problem's
    iterate matches the FP64 oracle's k-th iterate from the same x0 within
    1e-4 of the problem's largest entry."""
    batch = 67
    D, O = _btd_spd(nb, N, batch, 360 + nb + N)
    r = W.rng(361)
    b = r.standard_normal(batch * N * nb).astype(np.float32)
    x0 = r.standard_normal(batch * N * nb).astype(np.float32)
    for k in ((1,) if N == 1 else (1, 2, 5)):  # one block: M = T, one iteration solves exactly
        want, wdone = oracle.btd_pcg(nb, N, D.astype(np.float64), O.astype(np.float64), b.astype(np.float64),
                                     x0.astype(np.float64), k, 0.0, batch)
        assert (wdone == k).all()
        for pack in (0, 1):
            st, X, done = _pcg(nb, N, D, O, b, x0, k, 0.0, batch, pack)
            assert st == g.GLASS_OK, g.status_string(st)
            assert (done == k).all(), (nb, N, k, pack)
            X, Wm = X.reshape(batch, -1), want.reshape(batch, -1)
            scale = np.abs(Wm).max(1, keepdims=True)
            assert (np.abs(X - Wm) <= 1e-4 * scale).all(), (nb, N, k, pack, np.max(np.abs(X - Wm) / scale))


@pytest.mark.parametrize("nb,N", [(6, 32), (12, 32), (16, 64)])
def test_btd_pcg_converges_to_the_direct_solution(nb, N):
    """With a tolerance the loop stops by itself; the result then matches
    the oracle's direct (dense Cholesky) solve within 1e-4 per problem, and
    the iteration count is within one of the oracle's PCG at the same
    tolerance (the last comparison can fall either side in FP32)."""
    batch = 37
    D, O = _btd_spd(nb, N, batch, 370 + nb)
    b = W.rng(371).standard_normal(batch * N * nb).astype(np.float32)
    x0 = np.zeros_like(b)
    direct, info = oracle.btd_posv(nb, N, D.astype(np.float64), O.astype(np.float64), b.astype(np.float64), batch)
    assert (info == 0).all()
    _, wdone = oracle.btd_pcg(nb, N, D.astype(np.float64), O.astype(np.float64), b.astype(np.float64),
                              x0.astype(np.float64), 500, 1e-6, batch)
    st, X, done = _pcg(nb, N, D, O, b, x0, 500, 1e-6, batch)
    assert st == g.GLASS_OK
    assert (done > 0).all() and (done < 500).all() and (np.abs(done - wdone) <= 1).all(), (done, wdone)
    X, Dm = X.reshape(batch, -1), direct.reshape(batch, -1)
    assert (np.abs(X - Dm) <= 1e-4 * np.abs(Dm).max(1, keepdims=True)).all()


def test_btd_pcg_edge_cases():
    """iters = 0 leaves x; a non-SPD diagonal block gives -1 and leaves x; a
    short workspace is refused before any launch."""
    nb, N, batch = 3, 4, 6
    D, O = _btd_spd(nb, N, batch, 380)
    b = np.ones(batch * N * nb, np.float32)
    x0 = W.rng(381).standard_normal(batch * N * nb).astype(np.float32)
    st, X, done = _pcg(nb, N, D, O, b, x0, 0, 0.0, batch)
    assert st == g.GLASS_OK and (done == 0).all() and np.array_equal(X, x0)
    Dm = D.reshape(batch, N, nb, nb)
    Dm[2, 3] = -np.eye(nb, dtype=np.float32)
    st, X, done = _pcg(nb, N, D, O, b, x0, 5, 0.0, batch)
    assert st == g.GLASS_OK and done[2] == -1 and (np.delete(done, 2) == 5).all()
    assert np.array_equal(X.reshape(batch, -1)[2], x0.reshape(batch, -1)[2])
    st, _, _ = _pcg(nb, N, D, O, b, x0, 5, 0.0, batch, ws_bytes=g.glass_btd_pcg_workspace(nb, N, batch) - 4)
    assert st == g.GLASS_ERR_WORKSPACE
