"""GEMM with transposes and the LQR feedback gain on the GPU, through the C
ABI, against the FP64 oracle: every placement of the fused kernel and the
composition of primitive calls."""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W
from tests.helpers import U32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _padded(X, ld):
    """(batch, rows, cols) -> column-major with leading dimension ld (FP32)."""
    b, r, c = X.shape
    out = np.zeros((b, c, ld), dtype=np.float32)
    out[:, :, :r] = X.transpose(0, 2, 1)
    return out.reshape(-1), ld * c


GEMM_PL = [(g.GLASS_SCOPE_WARP, 1), (g.GLASS_SCOPE_WARP, 4), (g.GLASS_SCOPE_BLOCK, 1), (g.GLASS_SCOPE_BLOCK, 2)]


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(5, 7, 4), (33, 17, 64), (64, 64, 64), (1, 1, 1)])
def test_gemm_ex_matches_oracle(ta, tb, m, n, k):
    batch = 67
    r = W.rng(60 + m + 3 * n + 7 * k + 11 * ta + 13 * tb)
    A = r.standard_normal((batch, k, m) if ta else (batch, m, k)).astype(np.float32)
    B = r.standard_normal((batch, n, k) if tb else (batch, k, n)).astype(np.float32)
    C = r.standard_normal((batch, m, n)).astype(np.float32)
    a, sA = _padded(A, A.shape[1] + 1)
    b, sB = _padded(B, B.shape[1] + 2)
    c, sC = _padded(C, m + 3)
    lda, ldb, ldc = A.shape[1] + 1, B.shape[1] + 2, m + 3
    alpha, beta = 1.5, -0.25
    want = oracle.gemm_ex(ta, tb, m, n, k, alpha, a, lda, sA, b, ldb, sB, beta, c.astype(np.float64), ldc, sC, batch)
    opA = np.abs(A.transpose(0, 2, 1) if ta else A).astype(np.float64)
    opB = np.abs(B.transpose(0, 2, 1) if tb else B).astype(np.float64)
    bound = (k + 2) * 2 * U32 * (abs(alpha) * opA @ opB + abs(beta) * np.abs(C))
    for scope, pack in GEMM_PL:
        dC = _dev(c)
        st = g.glass_batched_gemm_ex(ta, tb, m, n, k, alpha, _dev(a), lda, sA, _dev(b), ldb, sB, beta, dC, ldc, sC,
                                     batch, g.make_opts(scope=scope, pack=pack))
        g.check(st, f"gemm_ex {ta}{tb} {m}x{n}x{k} {scope}x{pack}")
        got = _host(dC).astype(np.float64)
        # padding rows of C are untouched
        assert np.array_equal(got.reshape(batch, n, ldc)[:, :, m:], c.reshape(batch, n, ldc)[:, :, m:])
        err = np.abs(got - want).reshape(batch, n, ldc).transpose(0, 2, 1)[:, :m]
        assert (err <= bound + 1e-30).all(), (ta, tb, m, n, k, scope, pack)


def test_gemm_ex_integer_bit_exact_and_beta_zero_ignores_c():
    batch, m, n, k = 40, 24, 9, 31
    r = W.rng(70)
    A = r.integers(-4, 5, size=(batch, k, m)).astype(np.float32)   # stored k x m, used transposed
    B = r.integers(-4, 5, size=(batch, k, n)).astype(np.float32)
    dC = _dev(np.full(batch * m * n, np.nan, dtype=np.float32))
    g.check(g.glass_batched_gemm_ex(1, 0, m, n, k, 1.0, _dev(W.colmajor(A)), k, k * m, _dev(W.colmajor(B)), k,
                                    k * n, 0.0, dC, m, m * n, batch))
    got = W.from_colmajor(_host(dC), batch, m, n)
    assert np.array_equal(got, A.transpose(0, 2, 1) @ B)


def _riccati_ref(nx, nu, A, B, P, R, batch):
    K, info = oracle.riccati_gain(nx, nu, A.astype(np.float64), B.astype(np.float64), P.astype(np.float64),
                                  R.astype(np.float64), batch)
    return K, info


def _fused_placements(nx, nu):
    out = []
    for scope in (g.GLASS_SCOPE_WARP, g.GLASS_SCOPE_BLOCK):
        for pack in (1, 2, 4, 8):
            if g.glass_riccati_feasible(nx, nu, scope, pack):
                out.append((scope, pack))
    return out


def _run_riccati(nx, nu, A, B, P, R, batch, scope, pack, ws=True):
    import torch
    dK = torch.full((batch * nu * nx,), float("nan"), device="cuda")
    info = torch.full((batch,), -7, dtype=torch.int32, device="cuda")
    wsb = g.glass_riccati_workspace(nx, nu, batch) if ws else 0
    wst = torch.empty(max(1, wsb), dtype=torch.uint8, device="cuda")
    st = g.glass_riccati_gain(nx, nu, _dev(A), nx * nx, _dev(B), nx * nu, _dev(P), nx * nx, _dev(R), nu * nu,
                              dK, nu * nx, info, batch, wst if ws else None, wsb,
                              g.make_opts(scope=scope, pack=pack))
    return st, dK, info


@pytest.mark.parametrize("nx,nu", W.RICCATI_SIZES + [(1, 1), (33, 5), (64, 64)])
def test_riccati_gain_every_placement_matches_oracle(nx, nu):
    batch = 131
    A, B, P, R = W.riccati_inputs(nx, nu, batch, 80 + nx + nu)
    K, info_ref = _riccati_ref(nx, nu, A, B, P, R, batch)
    assert (info_ref == 0).all()
    scale = np.abs(K).max()
    for scope, pack in _fused_placements(nx, nu) + [(g.GLASS_SCOPE_COMPOSED, 0)]:
        st, dK, info = _run_riccati(nx, nu, A, B, P, R, batch, scope, pack)
        g.check(st, f"riccati {nx}x{nu} {scope}x{pack}")
        got = _host(dK).astype(np.float64)
        assert (_host(info) == 0).all(), (nx, nu, scope, pack)
        assert np.abs(got - K).max() <= 1e-4 * scale, (nx, nu, scope, pack, np.abs(got - K).max() / scale)


def test_riccati_gain_dyadic_exact_and_auto():
    # B = P = I, R = 3 I: S = 4 I, K = A / 4 exactly on every path
    nx = nu = 12
    batch = 70
    A = W.rng(90).integers(-8, 9, size=(batch, nx, nx)).astype(np.float64)
    I = np.broadcast_to(np.eye(nx), (batch, nx, nx))
    args = [W.colmajor(A), W.colmajor(I), W.colmajor(I), W.colmajor(3 * I)]
    for scope, pack in _fused_placements(nx, nu) + [(g.GLASS_SCOPE_COMPOSED, 0), (g.GLASS_SCOPE_AUTO, 0)]:
        st, dK, info = _run_riccati(nx, nu, *args, batch, scope, pack)
        g.check(st)
        assert np.array_equal(W.from_colmajor(_host(dK), batch, nu, nx), A / 4), (scope, pack)


def test_riccati_gain_info_and_workspace_rules():
    nx, nu, batch = 3, 2, 33
    A = W.colmajor(np.broadcast_to(np.eye(nx), (batch, nx, nx)))
    B = np.zeros(batch * nx * nu, dtype=np.float32)
    P = W.colmajor(np.broadcast_to(np.eye(nx), (batch, nx, nx)))
    Rm = np.broadcast_to(np.eye(nu), (batch, nu, nu)).copy()
    Rm[::2] = [[1.0, 2.0], [2.0, 1.0]]              # even problems: S = R indefinite, second pivot fails
    R = W.colmajor(Rm)
    for scope, pack in [(g.GLASS_SCOPE_WARP, 1), (g.GLASS_SCOPE_BLOCK, 1), (g.GLASS_SCOPE_COMPOSED, 0)]:
        st, _, info = _run_riccati(nx, nu, A, B, P, R, batch, scope, pack)
        g.check(st)
        inf = _host(info)
        assert (inf[::2] == 2).all() and (inf[1::2] == 0).all(), (scope, pack)
    st, _, _ = _run_riccati(nx, nu, A, B, P, R, batch, g.GLASS_SCOPE_COMPOSED, 0, ws=False)
    assert st == g.GLASS_ERR_WORKSPACE
    # auto without workspace still runs (fused)
    st, _, info = _run_riccati(nx, nu, A, B, P, R, batch, g.GLASS_SCOPE_AUTO, 0, ws=False)
    g.check(st)
    assert (_host(info)[1::2] == 0).all()
