"""Parity at full size, in the launch configuration bench.py times: every
cell of the placement sweep at batch 16384 with the table's placement, the
mixed-size batch of 8192, the tensor-core GEMMs at batch 65536 and the
refined solve at batch 16384 -- each checked on sampled problems that the
oracle recomputes one by one (first, last and random indices)."""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W
from paper_2609_28179_gb300.cells import NPTS, OPS, SWEEP_N, Cell
from tests.helpers import U32, backward_error

pytestmark = pytest.mark.gpu

BATCH = 16384
SAMPLES = 24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


def _sample(batch, seed):
    idx = W.rng(seed).choice(batch, SAMPLES - 2, replace=False)
    return np.unique(np.concatenate([[0, batch - 1], idx]))


def _problem(t, b, per):
    return t[b * per:(b + 1) * per].cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("n", SWEEP_N)
def test_sweep_cell_full_batch_sampled(op, n):
    import torch
    cell = Cell(op, n, BATCH, sets=1, device_inputs=True, seed=5000 + n)
    inputs = {k: v.clone() for k, v in cell.pristine.items()}
    g.check(cell.launch(0), f"{op} n={n}")
    torch.cuda.synchronize()
    w = cell.work[0]
    k = cell.k
    for b in _sample(BATCH, 5100 + n):
        b = int(b)
        if op == "gemm":
            A, B = _problem(inputs["A"], b, n * n), _problem(inputs["B"], b, n * n)
            ref = oracle.gemm(n, n, n, A, B, 1)
            got = _problem(cell.out, b, n * n)
            bound = n * 2 * U32 * (np.abs(W.from_colmajor(A, 1, n, n)) @ np.abs(W.from_colmajor(B, 1, n, n)))
            assert (np.abs(W.from_colmajor(got - ref, 1, n, n)) <= bound + 1e-30).all(), (op, n, b)
        elif op == "posv":
            A, B = _problem(inputs["A"], b, n * n), _problem(inputs["B"], b, n)
            L, X, info = oracle.posv(n, 1, A, B, 1)
            assert int(cell.info[b]) == 0 and info[0] == 0
            x = _problem(w["B"], b, n)
            assert np.abs(x - X).max() <= 1e-4 * np.abs(X).max(), (op, n, b)
            Lg = np.tril(W.from_colmajor(_problem(w["A"], b, n * n), 1, n, n)[0])
            assert np.abs(Lg - np.tril(W.from_colmajor(L, 1, n, n)[0])).max() <= 1e-4 * np.abs(L).max()
        elif op == "trsm":
            L, B = _problem(inputs["A"], b, n * n), _problem(inputs["B"], b, n * k)
            X = oracle.trsm(n, k, L, B, 1)
            x = _problem(w["B"], b, n * k)
            assert np.abs(x - X).max() <= 1e-4 * np.abs(X).max(), (op, n, b)
        elif op == "getrf_getrs":
            A, B = _problem(inputs["A"], b, n * n), _problem(inputs["B"], b, n)
            LU, piv, X, info = oracle.getrf_getrs(n, 1, A, B, 1)
            assert int(cell.info[b]) == 0 and info[0] == 0
            gp = cell.ipiv[b * n:(b + 1) * n].cpu().numpy()
            # pivots are compared where the choice is unambiguous in FP32
            _, _, _, gap = oracle.getrf(n, A, 1)
            if gap[0] >= 1e-3:
                assert np.array_equal(gp, piv), (op, n, b)
            x = _problem(w["B"], b, n)
            Am = W.from_colmajor(A, 1, n, n)
            assert backward_error(Am, x.reshape(1, n, 1), B.reshape(1, n, 1)).max() <= 1e-4, (op, n, b)
            assert np.abs(x - X).max() <= 1e-4 * np.abs(X).max(), (op, n, b)
        elif op == "rot3":
            Rs = _problem(inputs["A"], b, 9 * k)
            ref = oracle.rot3_compose(k, Rs, 1)
            assert np.abs(_problem(cell.out, b, 9) - ref).max() <= 1e-5 * max(1, k / 8), (op, n, b)
        else:
            T, P = _problem(inputs["A"], b, 16 * k), _problem(inputs["B"], b, 3 * NPTS)
            ref = oracle.se3_apply(k, T, NPTS, P, 1)
            got = _problem(cell.out, b, 3 * NPTS)
            assert np.abs(got - ref).max() <= 1e-5 * max(1, k / 4) * np.abs(ref).max(), (op, n, b)


def test_plain_posv_n6_batch1024_full():
    import torch
    n, batch = 6, 1024
    A = W.spd(n, batch, 1000)
    b = W.gaussian(n * batch, 1001)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    g.check(g.glass_batched_posv(n, 1, dA, n, n * n, dB, n, n, info, batch,
                                 g.make_opts(scope=g.GLASS_SCOPE_THREAD, pack=1)))
    L, X, oinfo = oracle.posv(n, 1, A.astype(np.float64), b.astype(np.float64), batch)
    torch.cuda.synchronize()
    assert (info.cpu().numpy() == 0).all()
    x = dB.cpu().numpy().astype(np.float64)
    assert np.abs(x - X).max() <= 1e-4 * np.abs(X).max()


def test_mixed_size_8192_sampled():
    import torch
    batch, nrhs = 8192, 4
    sizes = W.varsize_sizes(batch, 1003)
    A, B, offA, offB = W.varsize_pack(sizes, nrhs, 1004)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    wsb = g.glass_posv_varsize_workspace(batch)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    g.check(g.glass_posv_varsize(batch, torch.from_numpy(sizes).cuda(), torch.from_numpy(offA).cuda(),
                                 torch.from_numpy(offB).cuda(), nrhs, dA, dB, info, ws, wsb, None))
    torch.cuda.synchronize()
    XA = dB.cpu().numpy().astype(np.float64)
    assert (info.cpu().numpy() == 0).all()
    for i in _sample(batch, 1005):
        i, n = int(i), int(sizes[i])
        _, X, _ = oracle.posv(n, nrhs, A[offA[i]:offA[i] + n * n].astype(np.float64),
                              B[offB[i]:offB[i] + n * nrhs].astype(np.float64), 1)
        assert np.abs(XA[offB[i]:offB[i] + n * nrhs] - X).max() <= 1e-4 * np.abs(X).max(), (i, n)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_tensor_core_gemm_65536_sampled(n):
    import torch
    batch = 65536
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5200 + n)
    A = torch.randn(batch * n * n, generator=gen, device="cuda")
    B = torch.randn(batch * n * n, generator=gen, device="cuda")
    C = torch.empty_like(A)
    o = g.make_opts(math=g.GLASS_MATH_3XTF32_TC)
    g.check(g.glass_batched_gemm(n, n, n, A, n, n * n, B, n, n * n, C, n, n * n, batch, o))
    torch.cuda.synchronize()
    for b in _sample(batch, 5300 + n):
        b = int(b)
        a, bb = _problem(A, b, n * n), _problem(B, b, n * n)
        ref = W.from_colmajor(oracle.gemm(n, n, n, a, bb, 1), 1, n, n)
        got = W.from_colmajor(_problem(C, b, n * n), 1, n, n)
        absab = np.abs(W.from_colmajor(a, 1, n, n)) @ np.abs(W.from_colmajor(bb, 1, n, n))
        assert (np.abs(got - ref) <= (2 * n * U32 + 2.0 ** -20) * absab + 1e-30).all(), (n, b)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_bf16_tensor_core_gemm_65536_sampled(n):
    """The BF16 mode at the bench's batch (order 64: two tcgen05 CTAs per SM,
    each walking about 215 problems through its pipeline): sampled products
    against the FP64 product of the bf16 operands, and a clear status word."""
    import torch
    batch = 65536
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5250 + n)
    A = torch.randn(batch * n * n, generator=gen, device="cuda").to(torch.bfloat16)
    B = torch.randn(batch * n * n, generator=gen, device="cuda").to(torch.bfloat16)
    C = torch.full((batch * n * n,), float("nan"), device="cuda")
    o = g.make_opts(dtype=g.GLASS_BF16, math=g.GLASS_MATH_BF16_TC)
    g.check(g.glass_batched_gemm(n, n, n, A, n, n * n, B, n, n * n, C, n, n * n, batch, o))
    assert g.glass_last_device_status() == g.GLASS_OK
    Af, Bf = A.float(), B.float()
    for b in _sample(batch, 5350 + n):
        b = int(b)
        a, bb = _problem(Af, b, n * n), _problem(Bf, b, n * n)
        ref = W.from_colmajor(oracle.gemm(n, n, n, a, bb, 1), 1, n, n)
        got = W.from_colmajor(_problem(C, b, n * n), 1, n, n)
        absab = np.abs(W.from_colmajor(a, 1, n, n)) @ np.abs(W.from_colmajor(bb, 1, n, n))
        assert (np.abs(got - ref) <= 2 * n * U32 * absab + 1e-30).all(), (n, b)


@pytest.mark.parametrize("n", [32, 64])
def test_refined_posv_16384_sampled(n):
    import torch
    base = W.kappa_spd(n, 64, 1e3, 5400 + n)
    A = np.tile(base, BATCH // 64)
    b = W.gaussian(n * BATCH, 5401 + n)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda()
    info = torch.zeros(BATCH, dtype=torch.int32, device="cuda")
    g.check(g.glass_batched_posv(n, 1, dA, n, n * n, dB, n, n, info, BATCH,
                                 g.make_opts(refine_steps=1, fp64_diag=1)))
    torch.cuda.synchronize()
    assert (info.cpu().numpy() == 0).all()
    for i in _sample(BATCH, 5402 + n):
        i = int(i)
        a, rhs = A[i * n * n:(i + 1) * n * n].astype(np.float64), b[i * n:(i + 1) * n].astype(np.float64)
        _, X, _ = oracle.posv(n, 1, a, rhs, 1)
        x = dB[i * n:(i + 1) * n].cpu().numpy().astype(np.float64)
        Am = W.from_colmajor(a, 1, n, n)
        assert backward_error(Am, x.reshape(1, n, 1), rhs.reshape(1, n, 1)).max() <= 1e-4
        assert np.abs(x - X).max() <= 1e-4 * np.abs(X).max(), (n, i)
