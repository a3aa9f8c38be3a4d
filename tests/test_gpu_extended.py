"""Parity of the precision path (tensor-core GEMM, FP64- and compensated-residual refinement),
the mixed-size persistent posv, and the learned cost model's kernels against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W
from tests.helpers import U32, backward_error, host, sync, to_dev, zeros_i32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


def mats(flat, batch, r, c):
    return W.from_colmajor(flat, batch, r, c)


def bf16_round(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def tf32_round(x):
    """Round to nearest (ties away) at 10 mantissa bits, as cvt.rna.tf32.f32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


# ------------------------------------------------------------ tensor cores
@pytest.mark.parametrize("n", [16, 32, 64])
@pytest.mark.parametrize("math", [g.GLASS_MATH_BF16_TC, g.GLASS_MATH_TF32_TC, g.GLASS_MATH_3XTF32_TC])
def test_tc_gemm_integer_bit_exact(n, math):
    import torch
    batch = 37
    A = W.colmajor(W.int_matrix(n, n, batch, 2000 + n))
    B = W.colmajor(W.int_matrix(n, n, batch, 2100 + n))
    ref = oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch)
    if math == g.GLASS_MATH_BF16_TC:
        dA = torch.from_numpy(A).to("cuda").to(torch.bfloat16)
        dB = torch.from_numpy(B).to("cuda").to(torch.bfloat16)
        o = g.make_opts(dtype=g.GLASS_BF16, math=math)
    else:
        dA, dB = to_dev(A), to_dev(B)
        o = g.make_opts(math=math)
    dC = to_dev(np.full(batch * n * n, np.nan, np.float32))
    g.check(g.glass_batched_gemm(n, n, n, dA, n, n * n, dB, n, n * n, dC, n, n * n, batch, o))
    sync()
    assert np.array_equal(host(dC).astype(np.float64), ref)


@pytest.mark.parametrize("n", [16, 24, 32])
def test_streaming_gemm_every_problem_of_a_large_batch(n):
    """The FP32 block placement of orders 16-32 runs the streaming split-TF32
    kernel, whose warps each walk several products (the next one's operands
    in flight): at batch 20011 -- more products than the grid has warps, and
    a ragged last round -- every product is checked, integer operands bit
    for bit and Gaussian ones at the FP32 bound against the FP64 oracle."""
    batch = 20011
    o = g.make_opts(scope=g.GLASS_SCOPE_BLOCK, pack=1)
    Ai = W.colmajor(W.int_matrix(n, n, batch, 2150 + n))
    Bi = W.colmajor(W.int_matrix(n, n, batch, 2160 + n))
    dC = to_dev(np.full(batch * n * n, np.nan, np.float32))
    g.check(g.glass_batched_gemm(n, n, n, to_dev(Ai), n, n * n, to_dev(Bi), n, n * n, dC, n, n * n, batch, o))
    sync()
    assert np.array_equal(host(dC).astype(np.float64),
                          oracle.gemm(n, n, n, Ai.astype(np.float64), Bi.astype(np.float64), batch))
    A = W.gaussian(batch * n * n, 2170 + n)
    B = W.gaussian(batch * n * n, 2180 + n)
    dC = to_dev(np.full(batch * n * n, np.nan, np.float32))
    g.check(g.glass_batched_gemm(n, n, n, to_dev(A), n, n * n, to_dev(B), n, n * n, dC, n, n * n, batch, o))
    sync()
    ref = mats(oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch), batch, n, n)
    got = mats(host(dC).astype(np.float64), batch, n, n)
    absab = np.abs(mats(A, batch, n, n).astype(np.float64)) @ np.abs(mats(B, batch, n, n).astype(np.float64))
    assert (np.abs(got - ref) <= 2 * n * U32 * absab + 1e-30).all(), n


@pytest.mark.parametrize("n", [16, 32, 64])
def test_tc_gemm_gaussian_errors(n):
    """BF16 and TF32 products match the FP64 product of the ROUNDED operands
    to FP32 accumulation accuracy; 3xTF32 meets the FP32 bound on the
    original operands (its error against FP64 is stated, 1e-4 bar)."""
    import torch
    batch = 301
    A = W.gaussian(batch * n * n, 2200 + n)
    B = W.gaussian(batch * n * n, 2300 + n)
    absAB = np.abs(mats(A, batch, n, n)) @ np.abs(mats(B, batch, n, n))
    for math in (g.GLASS_MATH_BF16_TC, g.GLASS_MATH_TF32_TC, g.GLASS_MATH_3XTF32_TC):
        if math == g.GLASS_MATH_BF16_TC:
            Ar, Br = bf16_round(A), bf16_round(B)
            dA = torch.from_numpy(A).to("cuda").to(torch.bfloat16)
            dB = torch.from_numpy(B).to("cuda").to(torch.bfloat16)
            o = g.make_opts(dtype=g.GLASS_BF16, math=math)
        else:
            Ar, Br = (tf32_round(A), tf32_round(B)) if math == g.GLASS_MATH_TF32_TC else (A, B)
            dA, dB = to_dev(A), to_dev(B)
            o = g.make_opts(math=math)
        ref = oracle.gemm(n, n, n, Ar.astype(np.float64), Br.astype(np.float64), batch)
        dC = to_dev(np.zeros(batch * n * n, np.float32))
        g.check(g.glass_batched_gemm(n, n, n, dA, n, n * n, dB, n, n * n, dC, n, n * n, batch, o))
        sync()
        C = mats(host(dC).astype(np.float64), batch, n, n)
        err = np.abs(C - mats(ref, batch, n, n)) / (absAB + 1e-30)
        # 3xTF32 drops the lo*lo term (<= 2^-22 relative) on top of FP32 accumulation
        bound = 2 * n * U32 + (2.0 ** -20 if math == g.GLASS_MATH_3XTF32_TC else 0.0)
        assert err.max() <= bound, (n, math, err.max(), bound)
        rel = np.linalg.norm((C - mats(oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch),
                                        batch, n, n)).reshape(batch, -1), axis=1) / (
            np.linalg.norm(mats(A, batch, n, n).reshape(batch, -1), axis=1) *
            np.linalg.norm(mats(B, batch, n, n).reshape(batch, -1), axis=1))
        if math == g.GLASS_MATH_3XTF32_TC:
            assert rel.max() <= 1e-4


# ------------------------------------------ fifth-generation tensor cores
@pytest.mark.parametrize("batch", [1, 2, 151, 152, 153, 457])
def test_umma_gemm64_batches_and_routes(batch):
    """Order 64: the FP32 block-scope placement (packed, aligned operands)
    and the 3xTF32 mode both run the persistent tcgen05 kernel -- one CTA
    per SM, problems strided by the grid, so batches around the SM count
    leave CTAs with 0, 1 or 2+ problems.  Both must meet the FP32 bound and
    agree bit for bit; no bounded wait may have given up."""
    n = 64
    A = W.gaussian(batch * n * n, 2500 + batch)
    B = W.gaussian(batch * n * n, 2600 + batch)
    ref = oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch)
    bound = n * 2 * U32 * (np.abs(mats(A, batch, n, n)) @ np.abs(mats(B, batch, n, n))) + 1e-30
    dA, dB = to_dev(A), to_dev(B)
    out = []
    for o in (g.make_opts(scope=2, pack=1), g.make_opts(math=g.GLASS_MATH_3XTF32_TC)):
        dC = to_dev(np.full(batch * n * n, np.nan, np.float32))
        g.check(g.glass_batched_gemm(n, n, n, dA, n, n * n, dB, n, n * n, dC, n, n * n, batch, o))
        assert g.glass_last_device_status() == g.GLASS_OK
        C = host(dC)
        assert (np.abs(mats(C.astype(np.float64) - ref, batch, n, n)) <= bound).all()
        out.append(C)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("batch", [303, 304, 305, 1000])
def test_umma_gemm64_bf16_batches_around_two_ctas_per_sm(batch):
    """BF16 order 64 runs two persistent tcgen05 CTAs per SM (grid
    min(batch, 2 x SMs)), so batches around and above 2 x 152 give CTAs one,
    two or many problems: the raw and tile stages are reused, the
    accumulator-free wait and the phase flips run.  Every product must match
    the FP64 product of the bf16-rounded operands to FP32 accumulation
    accuracy, and no bounded wait may have given up."""
    import torch
    n = 64
    A = W.gaussian(batch * n * n, 2800 + batch)
    B = W.gaussian(batch * n * n, 2900 + batch)
    Ar, Br = bf16_round(A), bf16_round(B)
    ref = mats(oracle.gemm(n, n, n, Ar.astype(np.float64), Br.astype(np.float64), batch), batch, n, n)
    bound = 2 * n * U32 * (np.abs(mats(Ar, batch, n, n)) @ np.abs(mats(Br, batch, n, n))) + 1e-30
    dA = torch.from_numpy(A).to("cuda").to(torch.bfloat16)
    dB = torch.from_numpy(B).to("cuda").to(torch.bfloat16)
    dC = to_dev(np.full(batch * n * n, np.nan, np.float32))
    o = g.make_opts(dtype=g.GLASS_BF16, math=g.GLASS_MATH_BF16_TC)
    g.check(g.glass_batched_gemm(n, n, n, dA, n, n * n, dB, n, n * n, dC, n, n * n, batch, o))
    assert g.glass_last_device_status() == g.GLASS_OK
    C = mats(host(dC).astype(np.float64), batch, n, n)
    assert (np.abs(C - ref) <= bound).all(), np.max(np.abs(C - ref) / bound)


def test_umma_gemm64_unaligned_operands_take_the_simt_kernel():
    """A 4-byte-offset operand cannot feed the bulk copies; the block-scope
    call still returns the FP32-accurate product (through the SIMT kernel)."""
    import torch
    n, batch = 64, 40
    A = W.gaussian(batch * n * n, 2700)
    B = W.gaussian(batch * n * n, 2701)
    ref = oracle.gemm(n, n, n, A.astype(np.float64), B.astype(np.float64), batch)
    bound = n * 2 * U32 * (np.abs(mats(A, batch, n, n)) @ np.abs(mats(B, batch, n, n))) + 1e-30
    bufA = torch.zeros(batch * n * n + 1, device="cuda")
    bufA[1:] = torch.from_numpy(A).cuda()
    dC = to_dev(np.zeros(batch * n * n, np.float32))
    g.check(g.glass_batched_gemm(n, n, n, bufA[1:], n, n * n, to_dev(B), n, n * n, dC, n, n * n, batch,
                                 g.make_opts(scope=2, pack=1)))
    assert g.glass_last_device_status() == g.GLASS_OK
    assert (np.abs(mats(host(dC).astype(np.float64) - ref, batch, n, n)) <= bound).all()


# -------------------------------------------------------------- refinement
@pytest.mark.parametrize("n", [8, 32, 64])
@pytest.mark.parametrize("kappa", [1e1, 1e3])
def test_refined_posv_improves_forward_error(n, kappa):
    batch = 96
    A = W.kappa_spd(n, batch, kappa, 2400 + n)
    b = W.gaussian(batch * n, 2401 + n)
    _, Xs, info_ref = oracle.posv(n, 1, A.astype(np.float64), b.astype(np.float64), batch)
    Am = mats(A, batch, n, n).astype(np.float64)
    scopes = [(1, 1), (2, 1)] + ([(0, 1)] if n <= 16 else [])
    for scope, pack in scopes:
        res = {}
        for refine in (0, 1):
            for fp64d in (0, 1):
                dA, dB, info = to_dev(A), to_dev(b), zeros_i32(batch)
                o = g.make_opts(scope=scope, pack=pack, refine_steps=refine, fp64_diag=fp64d)
                g.check(g.glass_batched_posv(n, 1, dA, n, n * n, dB, n, n, info, batch, o))
                sync()
                assert (host(info)[:batch] == 0).all()
                X = host(dB).astype(np.float64)
                fwd = np.abs(X - Xs).reshape(batch, n).max(1) / np.abs(Xs).reshape(batch, n).max(1)
                be = backward_error(Am, mats(X, batch, n, 1), mats(b, batch, n, 1).astype(np.float64))
                res[(refine, fp64d)] = (fwd, be)
                assert be.max() <= 1e-4, (n, kappa, scope, refine, be.max())
        f0, f1 = res[(0, 0)][0], res[(1, 0)][0]
        assert np.median(f1) <= np.median(f0), (n, kappa, scope, np.median(f0), np.median(f1))
        assert res[(1, 0)][1].max() <= res[(0, 0)][1].max() * 1.5 + 1e-7


@pytest.mark.parametrize("n", [5, 16, 32, 64])
@pytest.mark.parametrize("kappa", [1e1, 1e3, 1e6])
def test_dot2_residual_matches_the_fp64_residual(n, kappa):
    """The compensated FP32 residual (Dot2) is as accurate as one evaluated
    in twice the FP32 precision, about 2^-48 |A||x| against 2^-53 n |A||x|
    for FP64 accumulation: both are far below the FP32 rounding of x1, so
    the refined solutions of the two residuals agree to a few FP32 units of
    x1 at every conditioning, element by element -- and the Dot2 solve
    keeps the FP64 one's accuracy against the oracle (forward error no
    worse than the unrefined solve's, backward error within 1e-4)."""
    batch = 96
    A = W.kappa_spd(n, batch, kappa, 2460 + n)
    b = W.gaussian(batch * n, 2461 + n)
    _, Xs, _ = oracle.posv(n, 1, A.astype(np.float64), b.astype(np.float64), batch)
    Am = mats(A, batch, n, n).astype(np.float64)
    scopes = [(1, 1), (2, 1)] + ([(0, 1)] if n <= 16 else [])
    for scope, pack in scopes:
        X = {}
        for resid in (g.GLASS_RESIDUAL_FP64, g.GLASS_RESIDUAL_DOT2):
            dA, dB, info = to_dev(A), to_dev(b), zeros_i32(batch)
            o = g.make_opts(scope=scope, pack=pack, refine_steps=1, residual=resid)
            g.check(g.glass_batched_posv(n, 1, dA, n, n * n, dB, n, n, info, batch, o))
            sync()
            assert (host(info)[:batch] == 0).all()
            X[resid] = host(dB).reshape(batch, n).astype(np.float64)
        x64, xd2 = X[g.GLASS_RESIDUAL_FP64], X[g.GLASS_RESIDUAL_DOT2]
        scale = np.abs(x64).max(1, keepdims=True)
        assert (np.abs(xd2 - x64) <= 8 * 2.0 ** -24 * scale).all(), (n, kappa, scope, np.abs(xd2 - x64).max())
        be = backward_error(Am, xd2.reshape(batch, n, 1), mats(b, batch, n, 1).astype(np.float64))
        assert be.max() <= 1e-4, (n, kappa, scope, be.max())
        Xs2 = Xs.reshape(batch, n)
        f64 = np.abs(x64 - Xs2).max(1) / np.abs(Xs2).max(1)
        fd2 = np.abs(xd2 - Xs2).max(1) / np.abs(Xs2).max(1)
        assert np.median(fd2) <= 1.5 * np.median(f64) + 1e-7, (n, kappa, scope, np.median(f64), np.median(fd2))


def test_fp64_diag_reciprocal_is_the_rounded_fp64_value():
    """With fp64_diag the reciprocal of each Cholesky pivot is 1/sqrt(d) to
    FP64 accuracy rounded once to FP32.  A = [[d, 1], [1, 4d]] makes
    l21 = 1 * (1/l11), so L's (1, 0) entry exposes it: it must equal
    float(1 / sqrt(double(d))) for every problem but possibly a few at
    rounding boundaries (there within one ulp), and l11 = float(sqrt(d))."""
    import torch
    batch = 4099
    d = np.exp(W.rng(2350).uniform(-20, 20, batch)).astype(np.float32)
    A = np.zeros((batch, 2, 2), np.float32)
    A[:, 0, 0], A[:, 1, 0], A[:, 0, 1], A[:, 1, 1] = d, 1.0, 1.0, 4.0 * d
    want_r = (1.0 / np.sqrt(d.astype(np.float64))).astype(np.float32)
    want_l = np.sqrt(d.astype(np.float64)).astype(np.float32)
    for scope, pack in [(0, 1), (1, 1), (2, 1)]:
        dA, info = to_dev(W.colmajor(A)), zeros_i32(batch)
        g.check(g.glass_batched_potrf(2, dA, 2, 4, info, batch, g.make_opts(scope=scope, pack=pack, fp64_diag=1)))
        sync()
        L = host(dA).reshape(batch, 4)
        assert np.array_equal(L[:, 0], want_l), scope
        r = L[:, 1]
        ulps = np.abs(r.view(np.int32).astype(np.int64) - want_r.view(np.int32).astype(np.int64))
        assert ulps.max() <= 1 and (ulps > 0).sum() <= batch // 1000, (scope, int((ulps > 0).sum()))


# ----------------------------------------------------------- mixed sizes
@pytest.mark.parametrize("nrhs", [1, 4])
def test_varsize_posv_matches_oracle(nrhs):
    import torch
    batch = 777
    sizes = W.varsize_sizes(batch, 2500, lo=1, hi=64)
    A, B, offA, offB = W.varsize_pack(sizes, nrhs, 2501)
    dn = torch.from_numpy(sizes).cuda()
    doA = torch.from_numpy(offA).cuda()
    doB = torch.from_numpy(offB).cuda()
    dA, dB = to_dev(A), to_dev(B)
    info = zeros_i32(batch)
    wsb = g.glass_posv_varsize_workspace(batch)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    refs_in = [(A[offA[i]:offA[i] + int(sizes[i]) ** 2].astype(np.float64),
                B[offB[i]:offB[i] + int(sizes[i]) * nrhs].astype(np.float64)) for i in range(batch)]
    refs = {}
    for wpc in (0, 1, 4, 8):
        dA.copy_(torch.from_numpy(A))
        dB.copy_(torch.from_numpy(B))
        o = g.make_opts(scope=g.GLASS_SCOPE_WARP if wpc else g.GLASS_SCOPE_AUTO, pack=wpc)
        g.check(g.glass_posv_varsize(batch, dn, doA, doB, nrhs, dA, dB, info, ws, wsb, o))
        sync()
        assert (host(info)[:batch] == 0).all()
        LA, XA = host(dA).astype(np.float64), host(dB).astype(np.float64)
        for i in range(batch):  # every instance
            n = int(sizes[i])
            L, X, inf = oracle.posv(n, nrhs, refs_in[i][0], refs_in[i][1], 1) if i not in refs else refs[i]
            refs[i] = (L, X, inf)
            x = XA[offB[i]:offB[i] + n * nrhs]
            assert np.abs(x - X).max() <= 1e-4 * np.abs(X).max(), (i, n, wpc)
            l = np.tril(mats(LA[offA[i]:offA[i] + n * n], 1, n, n)[0])
            assert np.abs(l - np.tril(mats(L, 1, n, n)[0])).max() <= 1e-4 * np.abs(L).max(), (i, n, wpc)


def test_varsize_flags_bad_orders_and_failures_and_is_graph_capturable():
    import torch
    batch = 300
    sizes = W.varsize_sizes(batch, 2600, lo=6, hi=64)
    sizes[5] = 0
    sizes[17] = 65
    A, B, offA, offB = W.varsize_pack(np.clip(sizes, 1, 64), 1, 2601)
    # instance 40 is not SPD at its column 2
    n40 = int(sizes[40])
    A40 = A[offA[40]:offA[40] + n40 * n40].reshape(n40, n40)
    A40[2, 2] = -1.0
    dn = torch.from_numpy(sizes).cuda()
    doA, doB = torch.from_numpy(offA).cuda(), torch.from_numpy(offB).cuda()
    dA, dB = to_dev(A), to_dev(B)
    info = zeros_i32(batch)
    wsb = g.glass_posv_varsize_workspace(batch)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    # record into a CUDA graph, replay twice on fresh inputs
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=s):
        st = g.glass_posv_varsize(batch, dn, doA, doB, 1, dA, dB, info, ws, wsb, None)
    assert st == g.GLASS_OK
    for _ in range(2):
        dA.copy_(torch.from_numpy(A))
        dB.copy_(torch.from_numpy(B))
        info.fill_(99)
        graph.replay()
        sync()
        inf = host(info)[:batch]
        assert inf[5] == -1 and inf[17] == -1
        assert 1 <= inf[40] <= 3
        ok = np.ones(batch, bool)
        ok[[5, 17, 40]] = False
        assert (inf[ok] == 0).all()
    assert g.glass_last_device_status() == g.GLASS_OK


# ------------------------------------------------------------- cost model
DIN, H, DOUT = 8, 64, 12
NP = 5516


def _mlp_data(rows, seed):
    gg = W.rng(seed)
    w = (gg.standard_normal(NP) * 0.2).astype(np.float32)
    X = gg.standard_normal((rows, DIN)).astype(np.float32)
    T = gg.standard_normal((rows, DOUT)).astype(np.float32)
    M = (gg.random((rows, DOUT)) > 0.25).astype(np.float32)
    return w, X, T, M


@pytest.mark.parametrize("rows", [1, 63, 64, 257, 5000])
def test_mlp_forward_and_gradient_vs_oracle(rows):
    import torch
    w, X, T, M = _mlp_data(rows, 2700 + rows)
    dw, dX, dT, dM = to_dev(w), to_dev(X.reshape(-1)), to_dev(T.reshape(-1)), to_dev(M.reshape(-1))
    dY = to_dev(np.zeros(rows * DOUT, np.float32))
    g.check(g.glass_mlp_forward(DIN, dw, rows, dX, dY))
    Yref = oracle.mlp_fwd(DIN, H, DOUT, w.astype(np.float64), X.astype(np.float64))
    sync()
    Y = host(dY).reshape(rows, DOUT)
    assert np.abs(Y - Yref).max() <= 1e-4 * max(1.0, np.abs(Yref).max())
    wsb = g.glass_mlp_workspace(rows)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    dg = to_dev(np.zeros(NP, np.float32))
    dl = to_dev(np.zeros(1, np.float32))
    g.check(g.glass_mlp_loss_grad(DIN, dw, rows, dX, dT, dM, dg, dl, ws, wsb))
    loss_ref, grad_ref = oracle.mlp_loss_grad(DIN, H, DOUT, w.astype(np.float64), X.astype(np.float64),
                                              T.astype(np.float64), M.astype(np.float64))
    sync()
    assert abs(float(host(dl)[0]) - loss_ref) <= 1e-4 * abs(loss_ref)
    gr = host(dg).astype(np.float64)
    # element by element, each parameter block (W1 b1 W2 b2 W3 b3) against its
    # own scale: |g - g*| <= 1e-4 max(|g*|, 0.01 max_block |g*|) -- the floor
    # covers entries whose row sums cancel to far below their terms
    for lo, hi in ((0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 5504), (5504, 5516)):
        gs, rs = gr[lo:hi], grad_ref[lo:hi]
        tol = 1e-4 * np.maximum(np.abs(rs), 0.01 * np.abs(rs).max()) + 1e-30
        assert (np.abs(gs - rs) <= tol).all(), (rows, lo, np.max(np.abs(gs - rs) / tol))


def test_mlp_adam_matches_oracle_step():
    w, _, _, _ = _mlp_data(1, 2800)
    gr = W.gaussian(NP, 2801)
    m0 = (W.gaussian(NP, 2802) * 0.1).astype(np.float32)
    v0 = np.abs(W.gaussian(NP, 2803)).astype(np.float32) * 0.01
    dw, dg, dm, dv = to_dev(w), to_dev(gr), to_dev(m0), to_dev(v0)
    g.check(g.glass_mlp_adam(NP, dw, dg, dm, dv, 3, 1e-3))
    wr, mr, vr = w.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64)
    oracle.adam_step(wr, gr.astype(np.float64), mr, vr, 3, lr=1e-3)
    sync()
    assert np.abs(host(dw) - wr).max() <= 1e-6
    assert np.abs(host(dm) - mr).max() <= 1e-6 and np.abs(host(dv) - vr).max() <= 1e-6


@pytest.mark.parametrize("n", [24, 40, 64])
def test_tensor_core_paths_with_padded_leading_dimensions(n):
    """The blocked tensor-core kernels on operands that are not packed
    (lda > n, batch strides with slack: the 4-byte staging path) against
    the oracle on the same padded buffers; the padding stays untouched."""
    import torch
    batch, lda, ldb, nrhs = 70, n + 3, n + 1, 3
    sA, sB = lda * n + 5, ldb * nrhs + 2

    def pack(M, ld, s):
        out = np.full(batch * s, 7.0, dtype=np.float32)
        for b in range(batch):
            for j in range(M.shape[2]):
                out[b * s + j * ld: b * s + j * ld + M.shape[1]] = M[b, :, j]
        return out
    A = pack(W.from_colmajor(W.spd(n, batch, 1500 + n), batch, n, n), lda, sA)
    G = pack(W.from_colmajor(W.general(n, batch, 1501 + n), batch, n, n), lda, sA)
    B = pack(W.rng(1502 + n).standard_normal((batch, n, nrhs)), ldb, sB)
    f64 = lambda x: x.astype(np.float64)
    kw = dict(lda=lda, sA=sA, ldb=ldb, sB=sB)
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")

    _, Xr, ir = oracle.posv(n, nrhs, f64(A), f64(B), batch, **kw)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    g.check(g.glass_batched_posv(n, nrhs, dA, lda, sA, dB, ldb, sB, info, batch,
                                 g.make_opts(scope=g.GLASS_SCOPE_WARP, pack=2)))
    assert (info.cpu().numpy() == 0).all() and (ir == 0).all()
    assert np.abs(dB.cpu().numpy() - Xr).max() <= 1e-4 * np.abs(Xr).max()      # padding: 7 on both sides

    _, _, Xr, _ = oracle.getrf_getrs(n, nrhs, f64(G), f64(B), batch, **kw)
    dA, dB = torch.from_numpy(G).cuda(), torch.from_numpy(B).cuda()
    ipiv = torch.zeros(batch * n, dtype=torch.int32, device="cuda")
    g.check(g.glass_batched_getrf_getrs(n, nrhs, dA, lda, sA, ipiv, dB, ldb, sB, info, batch,
                                        g.make_opts(scope=g.GLASS_SCOPE_WARP, pack=2)))
    assert np.abs(dB.cpu().numpy() - Xr).max() <= 1e-4 * np.abs(Xr).max()

    Lp = pack(np.tril(W.from_colmajor(W.general(n, batch, 1503 + n), batch, n, n)) + n * np.eye(n), lda, sA)
    Xr = oracle.trsm(n, nrhs, f64(Lp), f64(B), batch, **kw)
    dB = torch.from_numpy(B).cuda()
    g.check(g.glass_batched_trsm(n, nrhs, torch.from_numpy(Lp).cuda(), lda, sA, dB, ldb, sB, batch,
                                 g.make_opts(scope=g.GLASS_SCOPE_BLOCK, pack=2)))
    assert np.abs(dB.cpu().numpy() - Xr).max() <= 1e-4 * np.abs(Xr).max()
