"""Robotics operations of the placement table on the GPU, through the C ABI,
at every placement, against the FP64 oracle (and, where results are not
unique, against the properties that are)."""
import numpy as np
import pytest

import oracle
import paper_2609_28179_gb300 as g
from paper_2609_28179_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BATCH = 333   # ragged against every CTA size
# argmax and softmax spread a problem over a warp or a 64-thread team; the
# element-wise operations (one problem's arithmetic is a short serial chain)
# are served at thread scope only
PLACEMENTS_TEAM = [(s, p) for s in (0, 1, 2) for p in (1, 2, 4, 8) if not (s == 2 and p == 8)]
PLACEMENTS = [(0, p) for p in (1, 2, 4, 8)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_28179_gb300 import _build
    _build.build()
    g.lib()


def _dev(x, dtype=np.float32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype)).cuda()


def _empty(n, dtype="float"):
    import torch
    return torch.full((n,), float("nan"), device="cuda") if dtype == "float" else \
        torch.full((n,), -1, dtype=torch.int32, device="cuda")


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64) if t.dtype != torch.int32 else t.cpu().numpy()


def _opts(s, p):
    return g.make_opts(scope=s, pack=p)


def test_quat_retract_and_error():
    q = W.unit_quaternions(BATCH, 200)
    d = W.rotation_vectors(BATCH, 201)
    ref = oracle.quat_retract(q.astype(np.float64), d.astype(np.float64), BATCH)
    for s, p in PLACEMENTS:
        out = _empty(4 * BATCH)
        g.check(g.glass_batched_quat_retract(_dev(q), _dev(d), out, BATCH, _opts(s, p)), f"retract {s}x{p}")
        assert np.abs(_host(out) - ref).max() <= 4e-7, (s, p)
    q2 = ref.astype(np.float32)
    err_ref = oracle.quat_error(q.astype(np.float64), q2.astype(np.float64), BATCH)
    for s, p in PLACEMENTS:
        out = _empty(3 * BATCH)
        g.check(g.glass_batched_quat_error(_dev(q), _dev(q2), out, BATCH, _opts(s, p)))
        got = _host(out)
        assert np.abs(got - err_ref).max() <= 2e-6, (s, p)
        # error of retract recovers the perturbation (to FP32 rounding of q2)
        assert np.abs(got - d).max() <= 5e-6, (s, p)


def test_quat_small_angles_and_identity():
    q = W.unit_quaternions(64, 202)
    for scale in (1e-4, 1e-8, 0.0):
        d = (scale * W.rotation_vectors(64, 203)).astype(np.float32)
        out = _empty(256)
        g.check(g.glass_batched_quat_retract(_dev(q), _dev(d), out, 64))
        ref = oracle.quat_retract(q.astype(np.float64), d.astype(np.float64), 64)
        assert np.abs(_host(out) - ref).max() <= 2.5e-7
        e = _empty(192)
        g.check(g.glass_batched_quat_error(_dev(q), _dev(q), e, 64))
        assert np.abs(_host(e)).max() <= 2e-7          # error(q, q) = 0


def test_se3_retract():
    T = W.se3_transforms(BATCH, 204).astype(np.float32)
    xi = W.twists(BATCH, 205).reshape(BATCH, 6)
    xi[:40] *= 1e-6                                     # small-angle branch
    xi[40:60, 3:] = 0.0                                 # pure translation
    xi = xi.reshape(-1)
    ref = oracle.se3_retract(T.astype(np.float64), xi.astype(np.float64), BATCH)
    for s, p in PLACEMENTS:
        out = _empty(16 * BATCH)
        g.check(g.glass_batched_se3_retract(_dev(T), _dev(xi), out, BATCH, _opts(s, p)))
        got = _host(out)
        assert np.abs(got - ref).max() <= 2e-6 * max(1.0, np.abs(ref).max()), (s, p)
        last = got.reshape(BATCH, 4, 4)[:, :, 3]        # bottom row (0 0 0 1)
        assert np.array_equal(last, np.tile([0.0, 0.0, 0.0, 1.0], (BATCH, 1)))


def test_motion_cross():
    r = W.rng(206)
    v, m = r.standard_normal(6 * BATCH).astype(np.float32), r.standard_normal(6 * BATCH).astype(np.float32)
    ref = oracle.motion_cross(v.astype(np.float64), m.astype(np.float64), BATCH)
    bound = 4 * 2.0 ** -24 * 2 * np.abs(v).max() * np.abs(m).max() * 2
    for s, p in PLACEMENTS:
        out = _empty(6 * BATCH)
        g.check(g.glass_batched_motion_cross(_dev(v), _dev(m), out, BATCH, _opts(s, p)))
        assert np.abs(_host(out) - ref).max() <= bound, (s, p)
    # integer inputs: exact
    vi, mi = r.integers(-8, 9, 6 * BATCH).astype(np.float32), r.integers(-8, 9, 6 * BATCH).astype(np.float32)
    out = _empty(6 * BATCH)
    g.check(g.glass_batched_motion_cross(_dev(vi), _dev(mi), out, BATCH))
    assert np.array_equal(_host(out), oracle.motion_cross(vi.astype(np.float64), mi.astype(np.float64), BATCH))


def test_eig3():
    A = W.sym3(BATCH, 207)
    w_ref, V_ref = oracle.eig3(A.astype(np.float64), BATCH)
    Am = A.reshape(BATCH, 3, 3).astype(np.float64)
    scale = np.abs(Am).max(axis=(1, 2))
    wr = w_ref.reshape(BATCH, 3)
    gap = np.minimum(wr[:, 1] - wr[:, 0], wr[:, 2] - wr[:, 1]) / scale
    for s, p in PLACEMENTS:
        w, V = _empty(3 * BATCH), _empty(9 * BATCH)
        g.check(g.glass_batched_eig3(_dev(A), w, V, BATCH, _opts(s, p)))
        wg = _host(w).reshape(BATCH, 3)
        Vg = _host(V).reshape(BATCH, 3, 3).transpose(0, 2, 1)     # column-major -> matrix
        assert (np.abs(wg - wr).max(axis=1) <= 4e-6 * scale).all(), (s, p)
        assert np.abs(Vg.transpose(0, 2, 1) @ Vg - np.eye(3)).max() <= 4e-6, (s, p)
        res = np.abs(Am @ Vg - Vg * wg[:, None, :]).max(axis=(1, 2))
        assert (res <= 8e-6 * scale).all(), (s, p)
        Vr = V_ref.reshape(BATCH, 3, 3).transpose(0, 2, 1)
        sep = gap > 1e-2                                # vectors are unique (with the sign rule) there
        assert np.abs(Vg[sep] - Vr[sep]).max() <= 1e-3, (s, p)


def test_svd3_and_closest_rotation():
    M = W.rng(208).standard_normal(9 * BATCH).astype(np.float32)
    Mm = M.reshape(BATCH, 3, 3).transpose(0, 2, 1).astype(np.float64)
    _, s_ref, _ = oracle.svd3(M.astype(np.float64), BATCH)
    R_ref = oracle.closest_rotation(M.astype(np.float64), BATCH)
    sr = s_ref.reshape(BATCH, 3)
    for s, p in PLACEMENTS:
        U, S, V = _empty(9 * BATCH), _empty(3 * BATCH), _empty(9 * BATCH)
        g.check(g.glass_batched_svd3(_dev(M), U, S, V, BATCH, _opts(s, p)))
        Ug = _host(U).reshape(BATCH, 3, 3).transpose(0, 2, 1)
        Vg = _host(V).reshape(BATCH, 3, 3).transpose(0, 2, 1)
        Sg = _host(S).reshape(BATCH, 3)
        assert (np.abs(Sg - sr).max(axis=1) <= 4e-6 * sr[:, 0]).all(), (s, p)
        assert np.abs(Ug.transpose(0, 2, 1) @ Ug - np.eye(3)).max() <= 4e-6, (s, p)
        assert np.abs(Vg.transpose(0, 2, 1) @ Vg - np.eye(3)).max() <= 4e-6, (s, p)
        rec = np.abs(Ug * Sg[:, None, :] @ Vg.transpose(0, 2, 1) - Mm).max(axis=(1, 2))
        assert (rec <= 8e-6 * sr[:, 0]).all(), (s, p)
        R = _empty(9 * BATCH)
        g.check(g.glass_batched_closest_rotation(_dev(M), R, BATCH, _opts(s, p)))
        Rg = _host(R)
        sep = (sr[:, 1] - sr[:, 2]) / sr[:, 0] > 1e-2   # unique and well conditioned there
        err = np.abs(Rg - R_ref).reshape(BATCH, 9).max(axis=1)
        assert (err[sep] <= 2e-4).all(), (s, p)
        Rm = Rg.reshape(BATCH, 3, 3)
        assert np.abs(np.linalg.det(Rm) - 1.0).max() <= 1e-5, (s, p)


def test_svd3_rank_deficient_and_rotation_fixed_point():
    M = np.zeros((4, 3, 3))
    M[0] = np.diag([3.0, 2.0, 0.0])
    M[1] = np.outer([1.0, 2.0, 2.0], [0.0, 3.0, 4.0])     # rank one
    M[2] = np.zeros((3, 3))
    M[3] = W.se3_transforms(1, 209).reshape(4, 4).T[:3, :3]
    Mc = W.colmajor(M)
    U, S, V = _empty(36), _empty(12), _empty(36)
    g.check(g.glass_batched_svd3(_dev(Mc), U, S, V, 4))
    Ug = _host(U).reshape(4, 3, 3).transpose(0, 2, 1)
    Sg = _host(S).reshape(4, 3)
    assert np.abs(Sg[0] - [3.0, 2.0, 0.0]).max() <= 1e-6
    assert np.abs(Sg[1] - [15.0, 0.0, 0.0]).max() <= 2e-5
    assert np.abs(Ug.transpose(0, 2, 1) @ Ug - np.eye(3)).max() <= 1e-5
    R = _empty(36)
    g.check(g.glass_batched_closest_rotation(_dev(Mc), R, 4))
    assert np.abs(_host(R)[27:] - Mc[27:]).max() <= 2e-6  # a rotation is its own closest rotation


@pytest.mark.parametrize("n", [1, 5, 16, 33, 64, 200])
def test_argmax_and_softmax(n):
    r = W.rng(210 + n)
    x = r.standard_normal(BATCH * (n + 3)).astype(np.float32)
    xm = x.reshape(BATCH, n + 3)
    if n >= 4:
        xm[7, 1] = xm[7, 3] = 9.0                          # a tie: the first index wins
    sx = n + 3
    idx_ref = oracle.argmax(n, x.astype(np.float64), BATCH, sx=sx)
    sm_ref = oracle.softmax(n, x.astype(np.float64), BATCH, sx=sx).reshape(BATCH, n)
    for s, p in PLACEMENTS_TEAM:
        idx = _empty(BATCH, "int")
        g.check(g.glass_batched_argmax(n, _dev(x), sx, idx, BATCH, _opts(s, p)), f"argmax {s}x{p}")
        assert np.array_equal(_host(idx), idx_ref), (n, s, p)
        y = _empty(BATCH * (n + 1))
        g.check(g.glass_batched_softmax(n, _dev(x), sx, y, n + 1, BATCH, _opts(s, p)))
        got = _host(y).reshape(BATCH, n + 1)
        assert np.abs(got[:, :n] - sm_ref).max() <= 2e-6 * max(1, n / 16), (n, s, p)
        assert np.isnan(got[:, n]).all()                   # gap untouched


def test_element_wise_operations_refuse_team_placements():
    """A warp or block placement would run an element-wise operation's short
    serial chain on one lane of the team: such placements are not offered."""
    for op in range(7):
        for s, p in [(1, 1), (1, 4), (2, 1), (2, 4)]:
            assert not g.glass_robo_feasible(op, 1, s, p)
        assert g.glass_robo_feasible(op, 1, 0, 1)
    for op in (7, 8):
        assert g.glass_robo_feasible(op, 16, 1, 1) and g.glass_robo_feasible(op, 16, 2, 4)
    q = _dev(W.unit_quaternions(8, 5))
    assert g.glass_batched_quat_retract(q, _dev(np.zeros(24)), _empty(32), 8, _opts(1, 1)) == g.GLASS_ERR_INVALID_VALUE
