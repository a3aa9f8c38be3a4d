"""The C ABI library loads, exports every declared symbol, and rejects bad
arguments synchronously (CPU only: no call here reaches a kernel)."""
import os
import re

import pytest

import paper_2609_28179_gb300 as g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glass.h")


@pytest.fixture(scope="module")
def L():
    from paper_2609_28179_gb300 import _build
    _build.build()
    return g.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(glass_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("glass_batched_gemm", "glass_batched_potrf", "glass_batched_potrs", "glass_batched_trsm",
                 "glass_batched_getrf_getrs", "glass_batched_se3_apply", "glass_batched_posv",
                 "glass_batched_rot3_compose", "glass_posv_varsize", "glass_get_placement"):
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(L):
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in g.exported_symbols(), name
        assert hasattr(g, name), name


def test_version_and_status_strings(L):
    assert "sm_103a" in g.glass_version()
    assert g.status_string(g.GLASS_ERR_WORKSPACE) == "GLASS_ERR_WORKSPACE"


BAD = 0x10  # never dereferenced: every call below fails validation first


@pytest.mark.parametrize("n,expect", [(0, g.GLASS_ERR_INVALID_VALUE), (-3, g.GLASS_ERR_INVALID_VALUE),
                                      (65, g.GLASS_ERR_UNSUPPORTED)])
def test_order_limits(L, n, expect):
    assert g.glass_batched_posv(n, 1, BAD, 64, 4096, BAD, 64, 64, BAD, 4, None, 0) == expect
    assert g.glass_batched_potrf(n, BAD, 64, 4096, BAD, 4, None, 0) == expect
    assert g.glass_batched_trsm(n, 1, BAD, 64, 4096, BAD, 64, 64, 4, None, 0) == expect
    assert g.glass_batched_getrf_getrs(n, 1, BAD, 64, 4096, BAD, BAD, 64, 64, BAD, 4, None, 0) == expect


def test_batch_zero_is_a_noop(L):
    assert g.glass_batched_posv(6, 1, None, 6, 36, None, 6, 6, None, 0, None, 0) == g.GLASS_OK
    assert g.glass_batched_gemm(4, 4, 4, None, 4, 16, None, 4, 16, None, 4, 16, 0, None, 0) == g.GLASS_OK


def test_bad_arguments(L):
    I = g.GLASS_ERR_INVALID_VALUE
    assert g.glass_batched_posv(6, 1, None, 6, 36, BAD, 6, 6, BAD, 4, None, 0) == I       # null A
    assert g.glass_batched_posv(6, 1, BAD, 5, 36, BAD, 6, 6, BAD, 4, None, 0) == I        # lda < n
    assert g.glass_batched_posv(6, 1, BAD, 6, 20, BAD, 6, 6, BAD, 4, None, 0) == I        # overlapping
    assert g.glass_batched_posv(6, 1, BAD, 6, 36, BAD, 6, 6, None, 4, None, 0) == I       # null info
    assert g.glass_batched_posv(6, -1, BAD, 6, 36, BAD, 6, 6, BAD, 4, None, 0) == I
    assert g.glass_batched_gemm(4, 4, 4, BAD, 3, 16, BAD, 4, 16, BAD, 4, 16, 2, None, 0) == I
    o = g.make_opts(scope=g.GLASS_SCOPE_THREAD, pack=3)
    assert g.glass_batched_posv(6, 1, BAD, 6, 36, BAD, 6, 6, BAD, 4, o, 0) == I           # pack 3
    o = g.make_opts(scope=g.GLASS_SCOPE_THREAD, pack=1)
    assert g.glass_batched_posv(40, 1, BAD, 40, 1600, BAD, 40, 40, BAD, 4, o, 0) == I     # infeasible
    o = g.make_opts(layout=7)
    assert g.glass_batched_posv(6, 1, BAD, 6, 36, BAD, 6, 6, BAD, 4, o, 0) == I
    assert g.glass_batched_rot3_compose(0, BAD, 9, BAD, 9, 4, None, 0) == I
    assert g.glass_batched_rot3_compose(65, BAD, 9, BAD, 9, 4, None, 0) == g.GLASS_ERR_UNSUPPORTED
    assert g.glass_batched_se3_apply(2, BAD, 32, 10, BAD, 30, BAD, 29, 4, None, 0) == I  # sQ < 3 npts
    assert g.glass_posv_varsize(4, BAD, BAD, BAD, 1, BAD, BAD, BAD, BAD, 8, None, 0) == g.GLASS_ERR_WORKSPACE


def test_tensor_core_gemm_shape_rules(L):
    o = g.make_opts(dtype=g.GLASS_BF16, math=g.GLASS_MATH_BF16_TC)
    assert g.glass_batched_gemm(24, 24, 24, BAD, 24, 576, BAD, 24, 576, BAD, 24, 576, 4, o, 0) == \
        g.GLASS_ERR_UNSUPPORTED
    o = g.make_opts(dtype=g.GLASS_F32, math=g.GLASS_MATH_BF16_TC)
    assert g.glass_batched_gemm(32, 32, 32, BAD, 32, 1024, BAD, 32, 1024, BAD, 32, 1024, 4, o, 0) == \
        g.GLASS_ERR_INVALID_VALUE


def test_placement_queries(L):
    for op in (g.GLASS_OP_GEMM, g.GLASS_OP_POSV, g.GLASS_OP_TRSM, g.GLASS_OP_GETRF_GETRS):
        for n in (3, 6, 7, 12, 14, 24, 32, 64, 5, 50):
            for batch in (1, 64, 1024, 16384, 100000):
                s, (scope, pack) = g.glass_get_placement(op, n, n if op == g.GLASS_OP_TRSM else 1, batch)
                assert s == g.GLASS_OK
                assert g.glass_placement_feasible(op, n, n if op == g.GLASS_OP_TRSM else 1, scope, pack)
    s, pl = g.glass_get_placement(g.GLASS_OP_SE3, 4, 7, 1024)
    assert s == g.GLASS_OK and g.glass_placement_feasible(g.GLASS_OP_SE3, 4, 7, *pl)
    assert g.glass_get_placement(g.GLASS_OP_POSV, 65, 1, 10)[0] == g.GLASS_ERR_UNSUPPORTED
    # feasibility gating (Sec. III-A): no thread-scope Cholesky above 16, LU above 12
    assert not g.glass_placement_feasible(g.GLASS_OP_POSV, 24, 1, 0, 1)
    assert g.glass_placement_feasible(g.GLASS_OP_POSV, 16, 1, 0, 1)
    assert not g.glass_placement_feasible(g.GLASS_OP_GETRF_GETRS, 14, 1, 0, 1)
    assert g.glass_placement_feasible(g.GLASS_OP_GETRF_GETRS, 64, 1, 1, 8)


def test_learned_model_rejects_bad_weights(L):
    import numpy as np
    assert g.glass_set_learned_model(np.zeros(10), np.zeros(8), np.ones(8)) == g.GLASS_ERR_INVALID_VALUE
    assert g.glass_set_learned_model(np.zeros(5516), np.zeros(8), np.zeros(8)) == g.GLASS_ERR_INVALID_VALUE


def test_interleaved_layout_is_thread_scope_only(L):
    o = g.make_opts(layout=g.GLASS_LAYOUT_INTERLEAVED32, scope=g.GLASS_SCOPE_WARP, pack=1)
    assert g.glass_batched_posv(6, 1, BAD, 6, 36, BAD, 6, 6, BAD, 4, o, 0) == g.GLASS_ERR_UNSUPPORTED
    o = g.make_opts(layout=g.GLASS_LAYOUT_INTERLEAVED32, scope=g.GLASS_SCOPE_BLOCK, pack=1)
    assert g.glass_batched_getrf_getrs(6, 1, BAD, 6, 36, BAD, BAD, 6, 6, BAD, 4, o, 0) == g.GLASS_ERR_UNSUPPORTED
    o = g.make_opts(layout=g.GLASS_LAYOUT_INTERLEAVED32)   # auto: no thread-scope kernel above n = 16
    assert g.glass_batched_posv(40, 1, BAD, 40, 1600, BAD, 40, 40, BAD, 4, o, 0) == g.GLASS_ERR_UNSUPPORTED


def test_gemm_ex_and_riccati_argument_rules(L):
    I, U = g.GLASS_ERR_INVALID_VALUE, g.GLASS_ERR_UNSUPPORTED
    ex = g.glass_batched_gemm_ex
    assert ex(2, 0, 4, 4, 4, 1.0, BAD, 4, 16, BAD, 4, 16, 0.0, BAD, 4, 16, 2, None, 0) == I           # trans flag
    assert ex(1, 0, 4, 5, 3, 1.0, BAD, 2, 12, BAD, 3, 15, 0.0, BAD, 4, 20, 2, None, 0) == I           # lda < k (A^T)
    assert ex(0, 1, 4, 5, 3, 1.0, BAD, 4, 12, BAD, 4, 15, 0.0, BAD, 4, 20, 2, None, 0) == I           # ldb < n (B^T)
    assert ex(0, 0, 65, 4, 4, 1.0, BAD, 65, 260, BAD, 4, 16, 0.0, BAD, 65, 260, 2, None, 0) == U
    assert ex(0, 0, 4, 4, 4, 1.0, None, 4, 16, None, 4, 16, 0.0, None, 4, 16, 0, None, 0) == g.GLASS_OK
    o = g.make_opts(scope=g.GLASS_SCOPE_THREAD, pack=1)
    assert ex(0, 0, 4, 4, 4, 1.0, BAD, 4, 16, BAD, 4, 16, 0.0, BAD, 4, 16, 2, o, 0) == I        # no thread scope
    rg = g.glass_riccati_gain
    assert rg(0, 1, BAD, 0, BAD, 0, BAD, 0, BAD, 0, BAD, 1, BAD, 2, None, 0, None, 0) == I
    assert rg(65, 1, BAD, 0, BAD, 0, BAD, 0, BAD, 0, BAD, 65, BAD, 2, None, 0, None, 0) == U
    assert rg(4, 2, BAD, 16, BAD, 8, BAD, 16, BAD, 4, BAD, 7, BAD, 2, None, 0, None, 0) == I                    # sK < nu*nx
    assert rg(4, 2, BAD, 16, BAD, 8, BAD, 16, BAD, 4, BAD, 8, None, 2, None, 0, None, 0) == I                   # null info
    o = g.make_opts(scope=g.GLASS_SCOPE_COMPOSED)
    assert rg(4, 2, BAD, 16, BAD, 8, BAD, 16, BAD, 4, BAD, 8, BAD, 2, None, 0, o, 0) == g.GLASS_ERR_WORKSPACE
    assert rg(4, 2, BAD, 16, BAD, 8, BAD, 16, BAD, 0, BAD, 8, BAD, 2, BAD, 1 << 20, o, 0) == g.GLASS_ERR_WORKSPACE
    assert rg(4, 2, None, 0, None, 0, None, 0, None, 0, None, 8, None, 0, None, 0, None, 0) == g.GLASS_OK
    assert g.glass_riccati_workspace(12, 4, 1000) >= 4 * 1000 * (12 * 4 + 4 * 4)
    assert g.glass_riccati_workspace(0, 4, 10) == 0


def test_riccati_placement_queries(L):
    from paper_2609_28179_gb300 import workloads as W
    for nx, nu in W.RICCATI_SIZES + [(1, 1), (64, 64), (20, 3)]:
        for batch in (1, 64, 1024, 16384, 100000):
            for ok in (True, False):
                s, (scope, pack) = g.glass_riccati_placement(nx, nu, batch, ok)
                assert s == g.GLASS_OK
                if scope == g.GLASS_SCOPE_COMPOSED:
                    assert ok
                else:
                    assert g.glass_riccati_feasible(nx, nu, scope, pack)
    assert not g.glass_riccati_feasible(64, 64, g.GLASS_SCOPE_WARP, 8)   # shared memory
    assert not g.glass_riccati_feasible(8, 8, g.GLASS_SCOPE_BLOCK, 4)    # 512 threads
    assert not g.glass_riccati_feasible(8, 8, g.GLASS_SCOPE_THREAD, 1)


def test_fp64_storage_argument_rules(L):
    o = g.make_opts(dtype=g.GLASS_F64, refine_steps=1)
    assert g.glass_batched_posv(6, 1, BAD, 6, 36, BAD, 6, 6, BAD, 4, o, 0) == g.GLASS_ERR_UNSUPPORTED
    o = g.make_opts(dtype=g.GLASS_F64, scope=g.GLASS_SCOPE_THREAD, pack=1)
    assert g.glass_batched_getrf_getrs(9, 1, BAD, 9, 81, BAD, BAD, 9, 9, BAD, 4, o, 0) == g.GLASS_ERR_INVALID_VALUE
    o = g.make_opts(dtype=g.GLASS_F64, scope=g.GLASS_SCOPE_BLOCK, pack=1)
    assert g.glass_batched_trsm(6, 2, BAD, 6, 36, BAD, 6, 12, 4, o, 0) == g.GLASS_ERR_INVALID_VALUE
    o = g.make_opts(dtype=g.GLASS_F64, layout=g.GLASS_LAYOUT_INTERLEAVED32)
    assert g.glass_batched_gemm(4, 4, 4, BAD, 4, 16, BAD, 4, 16, BAD, 4, 16, 4, o, 0) == g.GLASS_ERR_UNSUPPORTED


def test_refinement_residual_option_is_validated(L):
    for resid in (-1, 2, 7):
        o = g.make_opts(refine_steps=1, residual=resid)
        assert g.glass_batched_posv(6, 1, BAD, 6, 36, BAD, 6, 6, BAD, 4, o, 0) == g.GLASS_ERR_INVALID_VALUE
    o = g.make_opts(refine_steps=1, residual=g.GLASS_RESIDUAL_DOT2)
    assert g.glass_batched_posv(6, 1, BAD, 6, 36, BAD, 6, 6, BAD, 0, o, 0) == g.GLASS_OK   # empty batch


def test_selftest_wait_timeout_rejects_bad_arguments(L):
    assert g.glass_selftest_wait_timeout(BAD, BAD, BAD, 4, 0, 0) == g.GLASS_ERR_INVALID_VALUE
    assert g.glass_selftest_wait_timeout(BAD, BAD, BAD, 4, (1 << 31) + 1, 0) == g.GLASS_ERR_INVALID_VALUE
    assert g.glass_selftest_wait_timeout(BAD, BAD, BAD, -1, 100, 0) == g.GLASS_ERR_INVALID_VALUE
    assert g.glass_selftest_wait_timeout(None, BAD, BAD, 4, 100, 0) == g.GLASS_ERR_INVALID_VALUE
    assert g.glass_selftest_wait_timeout(BAD, BAD, BAD, 0, 100, 0) == g.GLASS_OK
